/*
 * tgms.h -- C ABI of libtgms: a two-grid preconditioned conjugate-gradient
 * solver for the lowest-order Raviart-Thomas / P0 mixed discretisation of
 * Darcy flow, -div(kappa grad p) = f, with an adaptive spectral (GMsFEM)
 * coarse space, for one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: Yang, Fu & Chung, "A two-grid preconditioner with an adaptive
 * coarse space for flow simulations in highly heterogeneous media"
 * (arXiv 1807.07220).  Each entry point below cites the section / equation
 * whose operation it performs.
 *
 * Conventions (all arrays x-fastest, row-major in y, FP64):
 *   - the domain is the unit square split into n x n square cells, h = 1/n;
 *     coarse blocks K_i are b x b cells (b divides n);
 *   - cell arrays (kappa, f, p): n*n entries, cell (i, j) at j*n + i;
 *   - ux: (n+1)*n normal velocities of the x-faces, face (i, j) at x = i h,
 *     y in [j h, (j+1) h], index j*(n+1) + i, positive along +x;
 *   - uy: n*(n+1) normal velocities of the y-faces, face (i, j) at y = j h,
 *     x in [i h, (i+1) h], index j*n + i, positive along +y;
 *   - bflux: 4n OUTWARD normal velocities on the boundary faces: left
 *     (j = 0..n-1), right (j), bottom (i = 0..n-1), top (i);
 *   - "psi vectors" (operator-level entry points): n*n stream-function
 *     values at the nodes (i h, j h), node (i, j) at j*n + i; entries with
 *     i == 0 or j == 0 are boundary nodes and must be zero (the nodes
 *     i == n or j == n are implicit zeros).  A divergence-free face field with
 *     no boundary flux is u_x(i,j) = (psi(i,j+1)-psi(i,j))/h,
 *     u_y(i,j) = -(psi(i+1,j)-psi(i,j))/h.
 *
 * Ownership: the caller owns every buffer it passes.  tg_setup copies what it
 * keeps; the handle owns its device memory until tg_destroy.  With
 * TG_PTR_HOST the solver copies host arrays to and from the device inside
 * the call; with TG_PTR_DEVICE all array pointers must be device pointers
 * (e.g. torch CUDA tensors).  Operator-level entry points always take device
 * pointers.  All work is issued on the stream given to tg_setup; entry points
 * return after synchronising that stream.
 *
 * Errors: every int-returning function returns TG_OK (0) or a negative
 * TG_ERR_* code and never aborts; tg_strerror gives a message.
 */
#ifndef TGMS_H
#define TGMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TG_OK                       0
#define TG_ERR_INVALID_ARG         -1  /* sizes, b does not divide n, kappa <= 0 or not finite, NULL */
#define TG_ERR_INCOMPATIBLE_SOURCE -2  /* |sum F - boundary outflow| > 1e-12 * (sum |F| + outflow) */
#define TG_ERR_BREAKDOWN           -3  /* PCG: p^T K p <= 0 or non-finite alpha/beta */
#define TG_ERR_MAXITER             -4  /* not converged in max_iter; outputs still written */
#define TG_ERR_DEVICE_TIMEOUT      -5  /* a bounded device-side wait expired */
#define TG_ERR_CUDA                -6  /* CUDA runtime error (launch, copy, no device) */
#define TG_ERR_OOM                 -7  /* device allocation failed */
#define TG_ERR_UNSUPPORTED         -8  /* valid but not implemented configuration */
#define TG_ERR_DEGENERATE_BASIS    -9  /* a coarse face has no selected function with net flux */

/* precision of the preconditioner (patch inverses, coarse basis tiles and
 * inner residuals); the outer PCG vectors, dot products, fine operator and
 * the coarse matrix are always FP64. */
#define TG_PREC_F64  0
#define TG_PREC_F32  1
#define TG_PREC_BF16 2   /* BF16 patch inverses, FP32 coarse tiles, FP32 arithmetic */
#define TG_PREC_F16  3   /* FP16 patch inverses, each row scaled by a power of two that puts its
                            largest magnitude in [2^14, 2^15) (the factor is undone after the row's
                            FP32 dot product); FP32 coarse tiles; FP32 arithmetic.  Same bytes as
                            BF16 with three more mantissa bits. */

#define TG_PTR_HOST   0
#define TG_PTR_DEVICE 1

#define TG_CYCLE_TWO_GRID 0
#define TG_CYCLE_ADDITIVE 1

#define TG_COARSE_GMSFEM 0   /* adaptive spectral space, Section 4.2 */
#define TG_COARSE_MSFEM  1   /* one MsFEM function per coarse face, eq. msfem */
#define TG_COARSE_RT0    2   /* coarse RT0 space */
#define TG_COARSE_LEARNED 3  /* spectral problem of Section 4.2 restricted to predicted
                                flux profiles (see "learned coarse basis" below) */

/* solver of the FP64 coarse system (Section 5: the coarse problem is solved
 * by a direct method).  Both are exact up to rounding. */
#define TG_COARSE_SOLVER_AUTO  0   /* nested dissection above 768 coarse unknowns, else dense; a
                                      space whose kappa tg_update_kappa changes with its basis kept
                                      turns to the dense inverse (low-rank updates) at that call */
#define TG_COARSE_SOLVER_DENSE 1   /* explicit dense inverse: one GEMV of D^2 entries per solve */
#define TG_COARSE_SOLVER_ND    2   /* one level of nested dissection by coarse block rows: rows of
                                      coarse nodes separate strips of block rows; interior blocks and
                                      the separator Schur complement kept as dense FP64 inverses, so a
                                      solve reads sum_t (n_t^2 + 2 n_t m_t) + NS^2 entries (n_t interior
                                      and m_t adjacent separator unknowns of strip t, NS separator
                                      unknowns) in four launches.  Needs at least 4 coarse blocks per
                                      side (else the dense inverse is used); with tg_update_kappa the
                                      factor is formed again instead of updated by low rank */

typedef struct tg_handle tg_handle;
typedef struct tg_mlp tg_mlp;

typedef struct tg_grid {
  int nx, ny;     /* fine cells per side; this release requires nx == ny */
  int bx, by;     /* fine cells per coarse block side; bx == by, 2 <= b <= 16, b divides
                     n and n / b >= 2 (a single coarse block has no coarse faces, so
                     the coarse space of Section 4 would be empty: TG_ERR_INVALID_ARG) */
  int overlap;    /* oversampling of K_i^+ in fine cells (Section 6: 2), 1..2.  0 is
                     rejected (TG_ERR_INVALID_ARG): without oversampling the nodes on
                     the coarse grid lines lie in no patch, and the preconditioner
                     is singular on the divergence-free space */
} tg_grid;

typedef struct tg_options {
  double eta;        /* smoother weight, eq. smooth (Section 6: 0.2) */
  int m1, m2;        /* pre / post smoothing steps (Section 6: 1, 1) */
  int precision;     /* TG_PREC_* */
  int flexible;      /* 1: flexible CG beta = -alpha (z, K p) / (r, z)_old */
  int max_iter;      /* PCG iteration cap */
  int pointer_mode;  /* TG_PTR_HOST or TG_PTR_DEVICE for tg_setup / tg_solve */
  int coarse_space;  /* TG_COARSE_* */
  int max_basis;     /* cap on functions kept per coarse face; 0 = no cap */
  int profile;       /* 0: tg_solve runs one instantiated CUDA graph (PCG loop in a
                        device-side while node); 1: host-driven loop with CUDA
                        events around every smoother launch (timings in tg_report) */
  /* TG_COARSE_LEARNED only: the k predicted whitened flux profiles per coarse
   * face (see "learned coarse basis" below) come from face_profiles (device,
   * FP32, nfaces x learned_k x b, profile j of face f at f*learned_k*b + j*b
   * + l, l the fine face along E_i) when it is not
   * NULL, else from the network `net` (k = its k).  learned_max_iter > 0:
   * tg_solve rebuilds the coarse space with the exact spectral problems and
   * solves again when the learned space needed more PCG iterations. */
  const tg_mlp* net;
  const float* face_profiles;
  int learned_k;
  int learned_max_iter;
  /* smoother tile shape: -1 = autotune at setup (time every shape on the
   * handle's own patch inverses, keep the fastest; where the dense inverses,
   * counted at two bytes an entry, exceed 1.5 times the L2, a mixed-precision
   * handle forms no dense inverses and picks between the band forms 7 and 9
   * only); 0 = 16-byte loads, 4 rows
   * per pass (2 for FP64 storage); 1 = 16-byte loads, 2 rows; 2 = 8-byte
   * loads, 4 rows; 3 = 8-byte loads, 2 rows; 4 = TMA bulk copies into a
   * shared-memory ring; 5 = shape 3 and 6 = shape 1 software-pipelined (the
   * next pass's rows are loaded while the current pass is reduced); 7 =
   * the band form: each local problem solved from its band Cholesky factor by
   * two triangular solves (the paper's direct subdomain solver), one warp per
   * patch, in the arithmetic precision (FP64 handles FP64, the others FP32);
   * 8 = the tensor cores: BF16 / FP16 inverses stored a second time as
   * 16 x 16 tiles in mma operand order, applied by mma.m16n8k16 to the
   * residual split into three BF16 / FP16 parts (24 significant bits), FP32
   * accumulation; 9 = the band form with FP32 factors read ahead through a
   * shared-memory ring (cp.async, 44 rows ahead instead of 16 in registers:
   * faster where fewer patches leave HBM bandwidth to spare).  FP64 storage
   * runs shape 0 for 1..3, 5, 6, 8 and shape 7 for 9; FP32 storage shape 0
   * for 8; FP16 storage shape 0 for 4.  Shapes 0..6 and 8 compute the same
   * product of the stored inverses; shapes 7 and 9 the same operator. */
  int smoother_shape;
  /* 1: launch the kernels of a solve with programmatic dependent launch
   * (each kernel's launch overlaps the tail of the one before it; it waits
   * for that kernel's completion before reading its results); 0: plain
   * stream order.  Same results either way.  Default 0: on GB300 the
   * overlap measured slower (+14 % per solve at 256^2, +22 % at 1024^2),
   * the early-launched CTAs competing with the one-wave grids. */
  int launch_overlap;
  /* TG_CYCLE_TWO_GRID: the two-grid cycle of Section 5 (m1 smoothing steps,
   * the coarse correction, m2 smoothing steps, the residual recomputed after
   * each); TG_CYCLE_ADDITIVE: the two-level Schwarz preconditioner
   * z = S r + P r (eqs. smooth, coarsepre) that Section 5 contrasts with it,
   * both parts applied to r itself (m1, m2 unused).  Default two-grid. */
  int cycle;
  /* tg_setup_batch only: 1 (default) = the right-hand sides of an instance
   * advance in lock step, in groups of up to 4 that share every read of the
   * patch inverses in the two smoothing sweeps (each chain keeps its own PCG
   * scalars and stops on its own; iteration counts are those of separate
   * solves); used with m1 = m2 = 1 and the two-grid cycle.  0 = every
   * right-hand side an independent chain. */
  int batch_lockstep;
  /* tg_setup_batch with TG_COARSE_LEARNED only: candidate networks (host
   * array of nnets handles, NULL entries skipped); each instance takes the
   * first whose block size equals its own (a network is trained for one
   * block size), TG_ERR_INVALID_ARG when none does.  NULL: every instance
   * takes `net`. */
  const tg_mlp* const* batch_nets;
  int batch_nnets;
  int coarse_solver;   /* TG_COARSE_SOLVER_*, for the preconditioner's coarse space and the coarse
                          RT0 system of the preprocessing alike */
} tg_options;

typedef struct tg_report {
  int iters;              /* PCG iterations (applications of the fine operator) */
  int converged;          /* 1 if ||C^T r|| <= rtol ||C^T r_0|| */
  double rel_residual;    /* final ||C^T r|| / ||C^T r_0|| */
  double cond_estimate;   /* Lanczos estimate of cond(M K) from the PCG coefficients */
  int coarse_dim;         /* velocity basis + coarse cells + 1 (the paper's "Dim") */
  int velocity_basis;     /* number of coarse velocity functions, sum of l_i */
  int coarse_unknowns;    /* size of the SPD coarse system actually factored */
  double max_div_error;   /* max over cells of |int_c div u - F_c| / max |F_c| */
  double preprocess_ms;   /* device time of Section 3 (inside tg_solve) */
  double pcg_ms;          /* device time of the PCG loop */
  double epilogue_ms;     /* device time of v = vbar + vtilde and the pressure */
  int kernel_launches;    /* kernels of this library launched by the call */
  int smoother_launches;  /* profile == 1: smoother launches timed ... */
  double smoother_ms;     /* ... and their summed device time */
  int graph;              /* 1 if the call ran as one CUDA graph */
  int snapshot_solves;    /* local block solves of the coarse-space setup (Section 4.1) */
  int fallback_faces;     /* TG_COARSE_LEARNED: faces that took the exact spectral problem */
  int learned_fallback;   /* 1 if this call rebuilt the space exactly (learned_max_iter) */
  int smoother_shape;     /* smoother tile shape in use */
  float shape_us[10];     /* autotuner: microseconds per smoother launch of each shape (0: not tried) */
  int refactored_patches; /* patch inverses computed by the handle's last setup or tg_update_kappa */
  int refactored_blocks;  /* coarse-block factors computed by the same call */
  int update_rank[2];     /* last tg_update_kappa: rank of the low-rank update of the
                             coarse inverse ([0]) and of the coarse RT0 inverse ([1]);
                             -1: recomputed in full */
  int operator_launches;  /* profile == 1: launches of the PCG operator kernel (p = z + beta p,
                             q = K p, alpha) timed ... */
  double operator_ms;     /* ... and their summed device time */
  int coarse_solver;      /* TG_COARSE_SOLVER_DENSE or _ND: the solver of the preconditioner's coarse system */
  double coarse_solve_mb; /* matrix megabytes (1e6 B) that one coarse solve reads */
} tg_report;

/* Fills *opt with the parameters of Section 6 (eta 0.2, m1 = m2 = 1), FP64,
 * standard CG, max_iter 1000, TG_PTR_DEVICE, GMsFEM, no cap, profile 0, no
 * network or profiles, learned_k 4, learned_max_iter 0, smoother_shape -1,
 * launch_overlap 0, cycle TG_CYCLE_TWO_GRID, batch_lockstep 1. */
int tg_default_options(tg_options* opt);

/* Step 2 of Section 5 (and the setup half of Section 3): builds everything
 * that depends only on kappa.
 *   kappa   n*n cell permeabilities (> 0, finite), host or device per opt;
 *   grid    geometry; eig_tol the eigenvalue tolerance of Section 4.2
 *           (functions with lambda < eig_tol kept, at least one per face);
 *   stream  cudaStream_t (NULL = legacy default stream).
 * Builds: oversampled patch inverses L_i^{+-1} (eq. smooth) in the requested
 * precision; per-block snapshot spaces (eq. snapshot_eqn); per-face spectral
 * problems (eqs. spectral_1, spectral_eqn); the coarse basis and the FP64
 * coarse matrix R_H L_h R_H^T (eq. coarsepre) and its inverse; the coarse RT0
 * matrix used by the preprocessing.  *out receives the handle. */
int tg_setup(const double* kappa, const tg_grid* grid, double eig_tol,
             const tg_options* opt, void* stream, tg_handle** out);

/* Steps 1, 3 and 4 of Section 5: preprocessing (Section 3, eq. subproblem),
 * PCG on the reduced problem (eq. reduced_fine_system) preconditioned by the
 * two-grid cycle (eqs. smooth, coarsepre), then v = vbar + vtilde and the
 * pressure.
 *   f      n*n cell-average source densities (F_c = h^2 f_c);
 *   bflux  4n outward boundary normal velocities, or NULL for no flow (the
 *          paper's case); sum F must equal the net outflow;
 *   rtol   stop when ||C^T r||_2 <= rtol ||C^T r_0||_2 (Section 6: 1e-7);
 *   ux, uy, p  outputs (p physical sign, zero mean, obtained by integrating
 *          the discrete Darcy law A u = B^T p along grid lines with
 *          least-squares row offsets);
 *   iters  may be NULL; rep may be NULL.
 * Returns TG_ERR_MAXITER (outputs written) if not converged. */
int tg_solve(tg_handle* h, const double* f, const double* bflux, double rtol,
             double* ux, double* uy, double* p, int* iters, tg_report* rep);

/* tg_solve from an initial guess (ux0, uy0) of the velocity, e.g. the
 * previous step of a time-dependent run: PCG starts from the stream function
 * of the guess minus the preprocessing field vbar (built by integrating its
 * x-face values up each node column, exact when the guess carries the same
 * divergence and boundary flux as the solution; uy0 is not read and may be
 * NULL).  rtol is relative to the residual of the zero guess, as in tg_solve,
 * so the stopping target is the same and a good guess saves iterations; a
 * guess already within it returns with 0 iterations.  Pointers follow
 * pointer_mode like tg_solve's. */
int tg_solve_warm(tg_handle* h, const double* f, const double* bflux, double rtol, const double* ux0,
                  const double* uy0, double* ux, double* uy, double* p, int* iters, tg_report* rep);

/* New permeability for an existing handle (time-dependent runs such as the
 * two-phase flow of Section 6.2, where the pressure equation's coefficient is
 * kappa times the total mobility): kappa (n*n, > 0; host or device per
 * pointer_mode) replaces the setup's.  The smoother's patch inverses and the
 * block factors are recomputed in place for the patches and blocks that hold
 * a cell whose 1/kappa changed (the others are bitwise what a fresh setup
 * would compute; tg_report's refactored_* count them).
 *   coarse = 0: keeps the coarse basis of the first setup (the paper keeps
 *     the initial multiscale space).  The Galerkin matrices are linear in
 *     1/kappa, so their inverses change by a symmetric update of rank |S|,
 *     S the basis functions whose support meets a changed cell; it is
 *     applied in O(D^2 |S|) (Sherman-Morrison-Woodbury), or the inverse is
 *     recomputed in full when |S| > min(1024, D/4), after 64 updates in a row
 *     or on a non-positive pivot (tg_report's update_rank: |S|, -1 = full);
 *     a nested-dissection factor is formed again in full under
 *     TG_COARSE_SOLVER_ND, and replaced by the dense inverse (formed in
 *     full once, then updated as above) under TG_COARSE_SOLVER_AUTO;
 *   coarse = 1: rebuilds the coarse space by the handle's method (spectral
 *     problems, MsFEM or the learned basis); the coarse RT0 inverse of the
 *     preprocessing is updated as for 0;
 *   coarse = 2: as 0 with both inverses recomputed in full.
 * Solves after the call use the new kappa.  TG_ERR_INVALID_ARG for another
 * value of coarse. */
int tg_update_kappa(tg_handle* h, const double* kappa, int coarse);

/* Frees all device memory of the handle.  NULL is allowed. */
void tg_destroy(tg_handle* h);

/* Static message for an error code. */
const char* tg_strerror(int code);

/* Failure detection (no counterpart in the paper).  Every wait of a kernel of
 * this library on device-side state (the TMA smoother's mbarriers) is bounded;
 * when a bound expires the kernel raises a device flag, drains its own copies
 * (bounded again) and returns, and the call returns TG_ERR_DEVICE_TIMEOUT with
 * the context still usable.  This probe exercises that path without a fault:
 * one warp waits, for at most 2^limit_log2 polls (0 <= limit_log2 <= 22), on
 * an mbarrier in shared memory that it completes itself first (complete != 0:
 * returns TG_OK) or that nothing completes (complete == 0: the bound expires,
 * returns TG_ERR_DEVICE_TIMEOUT).  stream: cudaStream_t; synchronises it.
 * Shares the flag with running solves: call it with no solve in flight. */
int tg_probe_bounded_wait(int complete, int limit_log2, void* stream);

/* ---- operator-level entry points (device pointers, psi vectors) ----------
 * These expose single steps of the PCG iteration for verification; they run
 * exactly the kernels tg_solve runs. */

/* Fine operator of the reduced problem in stream-function form:
 * out = C^T A_h C psi (A_h of eq. fine_system), in FP64 (precision 0) or
 * FP32 arithmetic (precision 1). */
int tg_apply_operator(tg_handle* h, const double* psi, double* out, int precision);

/* Smoother of eq. smooth applied to the stream-function residual
 * rho = C^T r: z = eta * sum_i E_i (K_i^+)^{-1} E_i^T rho, K_i^+ the
 * oversampled local operator, in the handle's precision. */
int tg_apply_smoother(tg_handle* h, const double* rho, double* z);

/* Coarse correction of eq. coarsepre in stream-function form:
 * z = Psi (Psi^T K Psi)^{-1} Psi^T rho, Psi spanning the divergence-free part
 * of the coarse space. */
int tg_apply_coarse(tg_handle* h, const double* rho, double* z);

/* The two-grid preconditioner (Section 5: m1 smoothing steps, one coarse
 * step, m2 smoothing steps, residual recomputed after each). */
int tg_apply_preconditioner(tg_handle* h, const double* rho, double* z);

/* Spectral data of the coarse space (Section 4.2), host arrays:
 * nsel[nfaces] functions kept per coarse face, lambda[nfaces*b] all
 * eigenvalues ascending.  Coarse faces are ordered vertical (x = I H,
 * I = 1..nc-1, J = 0..nc-1, J-major) then horizontal (y = J H, J = 1..nc-1,
 * I = 0..nc-1, J-major).  Any pointer may be NULL. */
int tg_coarse_info(tg_handle* h, int* nfaces, int* velocity_basis, int* nsel, double* lambda);

/* Preprocessing of Section 3 alone: writes vbar (face arrays, device
 * pointers) with B_h vbar = F_h and the given boundary flux. */
int tg_preprocess(tg_handle* h, const double* f, const double* bflux, double* ux, double* uy);

/* ---- batched solves ------------------------------------------------------
 * Many independent problems -- kappa realisations on grids of different sizes,
 * each with several right-hand sides -- solved by ONE CUDA graph launch whose
 * ninst * nrhs PCG chains (Section 5, Steps 1, 3, 4 each) run concurrently on
 * the device.  All instances share options and eigenvalue tolerance; device
 * pointers only (pointer_mode TG_PTR_DEVICE, profile 0). */
typedef struct tg_batch tg_batch;

/* Step 2 of Section 5 for every instance: kappa[i] (device, n_i * n_i) on
 * grids[i]; nrhs right-hand sides per instance.  The batch owns the handles.
 * With smoother_shape -1, the autotuner runs for the first instance of each
 * (nx, bx, overlap); the later ones take the tile shape it chose (the same
 * patches give the same launches), so their reports' shape_us stay 0. */
int tg_setup_batch(int ninst, const double* const* kappa, const tg_grid* grids, double eig_tol,
                   const tg_options* opt, int nrhs, void* stream, tg_batch** out);

/* Solves all ninst * nrhs problems; every array holds ninst * nrhs device
 * pointers, instance-major (entry i * nrhs + k).  bflux may be NULL (all no
 * flow) or hold NULL entries.  iters and status (per problem TG_OK or a
 * TG_ERR_* code) may be NULL.  Returns TG_OK if every problem converged, else
 * the most severe per-problem code. */
int tg_solve_batch(tg_batch* batch, const double* const* f, const double* const* bflux, double rtol,
                   double* const* ux, double* const* uy, double* const* p, int* iters, int* status);

/* Number of instances and right-hand sides per instance. */
int tg_batch_size(tg_batch* batch, int* ninst, int* nrhs);

/* Frees the batch and its handles.  NULL is allowed. */
void tg_destroy_batch(tg_batch* batch);

/* ---- learned coarse basis -------------------------------------------------
 * The paper selects the coarse functions of each coarse face E_i by a local
 * spectral problem over its snapshot space (Section 4.2, eqs. spectral_1,
 * spectral_eqn; snapshots of eq. snapshot_eqn, one per fine face e_l of E_i
 * with normal component delta_l).  A coefficient vector over the snapshots is
 * therefore the normal-velocity profile g of the function on e_0..e_{b-1}
 * (its "flux profile", l running along +y on a vertical edge, +x on a
 * horizontal one, normal +x / +y).  Predictions are made in whitened
 * coordinates y_l = a_l^{1/2} g_l, a_l the mean of the two adjacent cells'
 * 1/kappa (the diagonal of the a-form), in which the spectral problem is
 * symmetric.  A network maps log kappa around E_i to k such profiles; the
 * setup extends each to omega_i with one local solve per block (instead of
 * b), solves the spectral problem on their span (Rayleigh-Ritz), keeps the
 * Ritz pairs with lambda < eig_tol (at least one) and falls back to the exact
 * problem of the face when its smallest Ritz value is >= eig_tol, when no
 * predicted direction is kept, or when the kept functions carry no net flux.
 *
 * Network input of face E_i: log10(kappa)/3 rounded to bfloat16 on the
 * (b + 2) x (2b + 2) cells of omega_i plus a one-cell halo (cells outside the
 * domain take the nearest cell's value), rows along E_i, columns across it
 * (K^1 first); a horizontal edge is transposed onto that layout.
 * Network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, weights and hidden
 * activations bfloat16, accumulation FP32; output entry j*b + l is profile j
 * at fine face l.  Parameters are one FP32 vector, layout W1 (hidden x din,
 * row-major), b1, W2 (hidden x hidden), b2, W3 (dout x hidden), b3 with
 * din = (b + 2)(2b + 2), dout = k b.
 * Training loss per face: ||G G^T - Q Q^T||_F^2, G the b x k predicted
 * whitened profiles as columns, Q the label (orthonormal basis of the span of
 * the whitened profiles of the k eigenfunctions with the smallest
 * eigenvalues), mean over the batch;
 * Adam (beta 0.9, 0.999, eps 1e-8).  bfloat16 arrays are passed as uint16_t.
 * All array pointers are device pointers. */

/* Sizes of the network for block size b (2..16), k profiles (1..8) and
 * hidden width (1..4096): din, dout, number of FP32 parameters. */
int tg_mlp_shape(int b, int k, int hidden, int* din, int* dout, long long* nparam);

/* Creates a network with parameters `params` (device, FP32, nparam) and Adam
 * state zero; work runs on `stream`. */
int tg_mlp_create(int b, int k, int hidden, const float* params, void* stream, tg_mlp** out);

/* Copies the FP32 parameters out (device, nparam). */
int tg_mlp_params(const tg_mlp* net, float* params);

/* y (batch x dout, FP32) = network(x (batch x din, bfloat16)). */
int tg_mlp_forward(tg_mlp* net, int batch, const uint16_t* x, float* y);

/* Loss and gradient of one batch, parameters unchanged: x (batch x din,
 * bfloat16), q (batch x k x b, FP32 labels, vectors as rows); *loss (host)
 * the mean loss; grad (device, nparam FP32, parameter layout) may be NULL.
 * batch <= 4096. */
int tg_mlp_loss_grad(tg_mlp* net, int batch, const uint16_t* x, const float* q, double* loss, float* grad);

/* nsteps Adam steps with learning rate lr; step s uses the samples
 * order[s*batch .. s*batch+batch-1] (device int32 indices into the
 * nsamples rows of x and q).  loss_hist (device, nsteps FP32) may be NULL.
 * batch <= 4096. */
int tg_mlp_train(tg_mlp* net, int nsamples, const uint16_t* x, const float* q, const int* order, int nsteps,
                 int batch, float lr, float* loss_hist);

/* Frees the network.  NULL is allowed. */
void tg_mlp_destroy(tg_mlp* net);

/* Training data of one field: for every coarse face (order of tg_coarse_info)
 * the network input x (nfaces x din, bfloat16) and the label q (nfaces x k x
 * b, FP32) from the exact spectral problems of Section 4.2 with tolerance
 * eig_tol; nsel (nfaces, the exact selection counts) and lambda (nfaces x b)
 * may be NULL.  kappa (device, n*n), grid as in tg_setup. */
int tg_face_data(const double* kappa, const tg_grid* grid, double eig_tol, int k, void* stream,
                 uint16_t* x, float* q, int* nsel, double* lambda);

/* ---- two-phase flow (Section 6.2) ---------------------------------------
 * IMPES building blocks, water and oil, porosity 1, relative permeabilities
 * k_rw = s^2, k_ro = (1 - s)^2.  Cell arrays n*n device pointers; work on
 * `stream`, the calls return after synchronising it. */

/* kappa_out = kappa * lambda(s), lambda(s) = s^2/mu_w + (1-s)^2/mu_o the total
 * mobility (eq. mobility): the permeability of the IMPES pressure equation. */
int tg_total_mobility(const double* kappa, const double* s, int n, double mu_w, double mu_o, double* kappa_out,
                      void* stream);

/* One explicit upstream-weighted saturation step (eq. DisSatEq_Implicit
 * evaluated at s^n): s_out = s + dt/h^2 (h^2 f+ - sum over faces of
 * (u h) f_w(upstream) + f_w(s) h^2 f-), with (ux, uy) the face velocities of
 * the pressure solve (boundary faces included: inward flow there is water)
 * and f the cell source densities (f > 0 injects water, f < 0 produces at the
 * cell's fractional flow).  dt_fixed > 0 is used as the time step; otherwise
 * dt = cfl h^2 / (F_max sigma), F_max the largest total outflow of a cell
 * (outgoing face fluxes plus its sink) and sigma the largest slope of f_w on
 * [0, 1] (20001 samples).  *dt (host, may be NULL) receives the step.  s_out
 * must not alias s.  The CFL reduction uses a scratch array compiled into the
 * library: calls that overlap on a device must be serialised. */
int tg_transport_step(const double* s, const double* ux, const double* uy, const double* f, int n, double cfl,
                      double dt_fixed, double mu_w, double mu_o, double* s_out, double* dt, void* stream);

/* ---- allocation-free entry point --------------------------------------
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory -- processes whose device memory is owned by another
 * allocator (a framework's caching allocator or a fixed arena reserved at
 * start-up, where an outside cudaMalloc can fail or fragment it), and
 * latency-critical paths that must not take cudaMalloc's implicit device
 * synchronisation.  It needs no handle and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * Pressure recovery, the same computation as the pressure output of tg_solve:
 * with kappa (n*n, > 0), and a face velocity (ux, uy) in the layout above,
 * writes p (n*n, physical sign, zero mean) by integrating the discrete Darcy
 * law A u = B^T p along grid rows and fitting one offset per row to the
 * y-face equations in least squares.  All pointers are device pointers;
 * work runs on `stream` (cudaStream_t, NULL = legacy default stream) and the
 * call returns after synchronising it.  TG_ERR_CUDA reports a failed launch,
 * copy or synchronisation of this call; a launch error already pending in
 * the calling thread is left pending and not reported.
 *
 * Scratch: one statically sized device array compiled into the library
 * (about 20 MiB, held by every GPU that loads the library until the process
 * exits) serves grids up to n = 1024; larger n returns TG_ERR_UNSUPPORTED,
 * n < 2 or a NULL pointer TG_ERR_INVALID_ARG, kappa <= 0 or not finite
 * TG_ERR_INVALID_ARG (p is then unspecified).  Every call on a device shares
 * that array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address (a one-time set-up per device).
 * The call cannot be recorded in a stream capture (it reads its status on
 * the host and synchronises the stream): on a stream that is being captured
 * it returns TG_ERR_UNSUPPORTED before enqueuing anything, and the capture
 * stays valid. */
int tg_pressure_noalloc(const double* kappa, const double* ux, const double* uy, double* p, int n,
                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TGMS_H */
