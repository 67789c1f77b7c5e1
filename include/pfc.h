/*
 * pfc.h - C ABI of the GB300 (sm_103a) PFC stage solver.
 *
 * The library solves the linear systems of the Ros3Pw Rosenbrock stages of the
 * P2 finite-element phase-field-crystal (PFC2, H^-1 gradient flow) equation of
 * Praetorius & Voigt, "Development and Analysis of a Block-Preconditioner for
 * the Phase-Field Crystal Equation" (arXiv:1501.06852), with FGMRES(restart)
 * around the approximate-factorisation block preconditioner P_CH (Eq. 4.1 with
 * the Cahn-Hilliard Schur approximation of Section 4.2), whose steps are
 * Jacobi-PCG solves with M, M + delta K and M + sqrt(delta) K.
 *
 * Conventions shared by every entry point
 * - Unknowns per field: n = (2 side + 1)^dim P2 dofs of a structured mesh of
 *   [0, length]^dim (2D: each square cut into 2 triangles along the diagonal
 *   from (i, j) to (i+1, j+1); 3D: each cube cut into the 6 Kuhn tetrahedra).
 *   Dofs are numbered lexicographically on the half-spacing lattice, x fastest.
 *   With options.degree = 1 (P1) the dofs are the (side + 1)^dim mesh vertices,
 *   numbered the same way.  pfc_host_pattern and pfc_host_stencil describe P2.
 * - A state or stage vector has 3n doubles: [mu (n) | psi (n) | omega (n)]
 *   (the unknowns x = (mu, psi, omega) of Section 3).
 * - Every vector argument is a DEVICE pointer (cudaMalloc'd or from a framework
 *   allocator) to float64 data owned by the caller; the library never frees it.
 *   Pointers must stay valid until the call returns (the calls that read back a
 *   scalar synchronise the context stream before returning).
 * - All work is enqueued on the CUDA stream given to pfc_setup_mesh.
 * - No call aborts.  Errors return a status; pfc_last_error describes the most
 *   recent one.  After PFC_ERR_CUDA the context must be destroyed.
 * - A context is not thread safe; distinct contexts are independent.
 */
#ifndef PFC_H
#define PFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfc_ctx pfc_ctx;

typedef enum {
  PFC_OK = 0,
  PFC_ERR_INVALID = 1,        /* bad argument or call order */
  PFC_ERR_OOM = 2,            /* device allocation failed */
  PFC_ERR_CUDA = 3,           /* CUDA runtime error; context unusable */
  PFC_ERR_NOT_CONVERGED = 4,  /* iteration cap reached; outputs hold the last iterate */
  PFC_ERR_NONFINITE = 5,      /* NaN/Inf met in a reduction */
  PFC_ERR_TIMEOUT = 6         /* a device-side grid barrier gave up waiting */
} pfc_status;

/* Precision of the inner preconditioner solves (the outer FGMRES, its residuals,
 * Arnoldi/Givens and step control are always float64). */
typedef enum {
  PFC_PREC_FP64 = 0,          /* inner PCG in float64 */
  PFC_PREC_FP32 = 1,          /* inner PCG with float32 matrix values and vectors */
  PFC_PREC_FP16 = 2           /* float16 matrix values, float32 vectors and accumulation */
} pfc_precision;

typedef struct {
  double r;           /* model parameter r of Eq. (2.1) */
  double outer_tol;   /* FGMRES stop: ||b - A^R y||_2 <= outer_tol ||b||_2 */
  double inner_rtol;  /* PCG stop: ||r||_2 <= inner_rtol ||rhs||_2 (Table 2: 1e-3) */
  int restart;        /* FGMRES restart length (Section 7: 30); 1..40 */
  int max_outer;      /* cap on FGMRES iterations per stage solve */
  int max_inner;      /* cap on PCG iterations per inner solve */
  int precision;      /* pfc_precision */
  double step_atol;   /* step-size control tolerances (1e-3, 1e-3) */
  double step_rtol;
  double tau_max;     /* upper bound for the next time-step width */
  int blocks_per_sm;  /* persistent-kernel residency; 0 = as many as fit */
  int pcg_variant;    /* inner CG form (all give the same iterates in exact arithmetic):
                         0 textbook Jacobi-PCG (3 grid barriers per iteration),
                         1 pipelined Jacobi-PCG of Ghysels & Vanroose (1 barrier),
                         3 Chronopoulos-Gear Jacobi-PCG (2 barriers),
                         2 automatic: pipelined with float64 inner solves,
                         Chronopoulos-Gear with float32/float16 ones (the pipelined
                         recurrences drift there and cost outer iterations) */
  int inner_operator; /* inner matrices M, K, M + delta K, M + sqrt(delta) K in the
                         preconditioner: 0 assembled SELL-32 values with int32 column
                         indices; 1 structured stencils - on this mesh every row whose
                         elements all exist has the same entries as every other row of its
                         dof type, so those rows read neither values nor indices (the
                         other rows keep their assembled values) */
  int smem_window;    /* with structured stencils and float32/float16 inner solves, where the
                         inner SpMV reads its source vector:
                         0: global memory, each warp gathering for its own slices;
                         1: each block copies the rows its rows reach (its own rows plus the
                         stencil reach on both sides) into shared memory once per product,
                         when that window fits without lowering the grid's residency; same
                         results bit for bit as 0;
                         2: each block walks its rows in chunks of 1024, one row per thread,
                         and the chunk's source window (its lattice lines and two more on
                         each side; in 3D that band in the five planes around it) is
                         bulk-copied into one of two shared-memory buffers (cp.async.bulk
                         completing on an mbarrier) while the previous chunk is computed;
                         the Chronopoulos-Gear inner solves use it (the per-row sums are
                         the same, the partial inner products are added in another order).
                         Chunks that cross a 3D plane boundary read global memory. */
  int model;          /* 2: PFC2, the H^-1 gradient flow of Eq. (2.2) (mobility 1);
                         1: PFC1, the Wasserstein flow of Eq. (2.3) with mobility
                         psi^+ = psi - psi_min: the second block row of the stage
                         system (Eq. 3.10) becomes [tau K_+(psi_k), M / gamma +
                         tau F(mu_k), 0] with K_+(psi) = ((psi^+ grad phi_j, grad phi_i))
                         and F(mu) = ((phi_j grad mu, grad phi_i)), b1 uses
                         -tau K_+(psi_i) mu_i, and P_CH takes the constant-mobility
                         approximation K_+ ~ M0 K of Section 4, M0 = <psi_k^+>
                         (its assembly reads M0 back: one extra synchronisation).
                         The Euler system keeps the mobility explicit:
                         [tau K_+(psi_k), M, 0]. */
  double psi_min;     /* PFC1: lower bound psi_min of the density (-1.5, Section 2) */
  int schur;          /* Schur-complement approximation in step (3) of the preconditioner:
                         0: S_CH of Section 4.2, steps (3.1) and (3.2);
                         1: S_D = M - 2 delta K + delta K M_D^{-1} K, M_D = diag(M)
                         (Section 4.1), one Jacobi-PCG solve of schur_its iterations
                         (Table 2: 20), applied without forming K M_D^{-1} K */
  int schur_its;      /* fixed PCG iterations of the S_D step (>= 1) */
  int degree;         /* Lagrange degree of V_h (Section 3): 2 (P2, default) or 1 (P1,
                         dofs on the mesh vertices, n = (side + 1)^dim per field) */
  double err_tol;     /* > 0: a stage solve also stops only once its estimated relative
                         solution error ||y - y*|| / ||y|| is at most err_tol; 0: the
                         residual test alone.  The paper fixes no outer tolerance
                         (Section 7); the stage solution is wanted to a relative error,
                         and the ratio of error to residual grows with tau as the stage
                         matrix of Eq. (3.10) nears the singularity of Lemma 3 (four
                         orders of magnitude at 0.9 tau*).  With right preconditioning
                         y - y* = P^{-1} (A^R P^{-1})^{-1} r, so once the residual test
                         passes the solver estimates E = ||P^{-1} r|| / (||y|| sigma),
                         sigma = the smallest singular value of the Hessenberg matrices
                         of its restart cycles so far, stops if E <= err_tol and otherwise
                         tightens its residual target to (||r|| / ||b||)(err_tol / E) / 2.
                         The ratio E / (||r|| / ||b||) of a context's last tested solve sets
                         the starting residual target of its next solve (scaled by the
                         ratio of the widths tau).  Default 1e-9. */
  double tau_guard;   /* > 0 (PFC2 only): pfc_step caps the next width so that gamma tau <=
                         tau_guard tau*(r, <psi>), tau* the critical width of Lemma 3 at the
                         mean density <psi> of the state (conserved by the flow); must be
                         < 1; 0 (default): no cap beyond tau_max */
  int grid_blocks;    /* > 0: the persistent solver of this context always runs on exactly
                         min(grid_blocks, its 32-row slices, co-resident blocks) blocks, alone
                         and in every batched launch, so its row partition and reduction
                         order, hence its results bit for bit, do not depend on what else
                         is in a batch (serving); 0 (default): alone it takes every
                         co-resident block, in a batch a share proportional to its rows */
  int cells;          /* P2 with structured stencils (inner_operator 1) and float32/float16
                         inner solves in the Chronopoulos-Gear form: 1 (default) numbers
                         the rows by 2 x 2 (2D) or 2 x 2 x 2 (3D) lattice cells (a cell's
                         dofs are consecutive rows, so a vector moves four of them per
                         16-byte access), and the inner solves run one grid barrier per
                         iteration: every block owns a tile of cells and keeps u on it
                         and on the ring of cells around it in shared memory, recomputing
                         the ring from its neighbours' r, s, w rather than waiting for
                         them (same iterates in exact arithmetic); when the tile's window
                         does not fit in shared memory the context keeps the
                         lexicographic rows; 0: the lexicographic order.  Ignored
                         elsewhere (float64, P1, assembled inner matrices). */
} pfc_options;

typedef struct {
  int outer_its;        /* FGMRES iterations */
  int restarts;         /* completed restart cycles */
  long long inner_its;  /* total PCG iterations over all preconditioner applications */
  int inner_calls;      /* number of PCG solves */
  int inner_capped;     /* PCG solves that hit max_inner */
  double rel_residual;  /* final true ||b - A^R y||_2 / ||b||_2, recomputed in float64 */
  int status;           /* pfc_status of this solve */
  double phase_ms[8];   /* with pfc_set_timing on: block 0's time in [inner SpMV phases,
                           inner vector phases, outer FGMRES phases, PCG set-up phases]
                           (work), then the same four classes of barrier waits */
  double err_est;       /* the solution-error estimate E of the last test (options.err_tol);
                           NaN when no test ran */
  double sigma_min;     /* smallest singular value of the restart cycles' Hessenberg
                           matrices (estimate of that of A^R P^{-1}); inf when none */
} pfc_solve_stats;

/* Fills the defaults: r = -0.4, outer_tol = 1e-10, inner_rtol = 1e-3,
 * restart = 30, max_outer = 600, max_inner = 1000, precision = FP64,
 * step_atol = step_rtol = 1e-3, tau_max = 1e9, blocks_per_sm = 0, pcg_variant = 2, inner_operator = 1,
 * smem_window = 0, model = 2, psi_min = -1.5, schur = 0, schur_its = 20, degree = 2,
 * err_tol = 1e-9, tau_guard = 0, grid_blocks = 0, cells = 1. */
void pfc_default_options(pfc_options* opt);

/* Critical time-step width of Lemma 3 (Section 6): the symbol of the PFC2 operator
 * linearised about the constant density psi_bar has the eigenvalue zero once the
 * effective width (gamma tau in a Rosenbrock stage) reaches
 *   tau* = 27 / (2 (sqrt(alpha) - 1)(sqrt(alpha) + 2)^2),  alpha = 1 - 3 r - 9 psi_bar^2.
 * Returns +infinity when alpha <= 1 (psi_bar^2 >= -r / 3: no critical width).
 * Host only; no context, no GPU. */
double pfc_critical_tau(double r, double psi_bar);

/* Mesh, P2 dof map, shared SELL-32 sparsity pattern of all blocks, and the
 * constant M and K (Section 3, the matrices below Eq. 3.4).  dim is 2 or 3,
 * side >= 1, length > 0.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  On success *out owns all device memory of the instance.  On failure
 * *out may still receive a context that holds only the error text: read it with
 * pfc_last_error and release it with pfc_destroy. */
pfc_status pfc_setup_mesh(pfc_ctx** out, int dim, int side, double length,
                          const pfc_options* opt, void* cuda_stream);

/* Dofs per field n of a set-up context (0 for NULL). */
int64_t pfc_num_dofs(const pfc_ctx* ctx);

/* Device bytes a context with these sizes would hold (for admission control). */
size_t pfc_footprint_bytes(int dim, int side, const pfc_options* opt);

/* Per-step assembly at the state x^k (3n, device): the (mu, psi) block
 * A01 = -(1+r) M + 2 K + N(psi^k), N(psi)_ij = (-3 psi^2 phi_j, phi_i)
 * (Eq. 3.10 with K_+ = K, F = 0 for PFC2), and for the step width tau the
 * inner matrices M + delta K and M + sqrt(delta) K with delta = sqrt(gamma tau)
 * and their Jacobi diagonals (Section 4, Table 2).  Must precede the stage
 * calls; the matrices stay until the next pfc_assemble. */
pfc_status pfc_assemble(pfc_ctx* ctx, const double* state, double tau);

/* Right-hand side b_i^R of Eq. (3.10) for stage i = nprev (0, 1 or 2) at the
 * stage value x_i (3n, device):
 *   b0 = -M mu_i + (1+r) M psi_i - 2 K psi_i - K omega_i + (psi_i^3, phi)
 *   b1 = -tau K mu_i + sum_{j<i} c_ij M dpsi_j
 *   b2 = -M omega_i - K psi_i
 * y_prev holds the nprev previous stage increments back to back (nprev x 3n,
 * device; may be NULL when nprev == 0); c_ij are the Ros3Pw coefficients of
 * Table 1.  Writes b (3n, device). */
pfc_status pfc_stage_rhs(pfc_ctx* ctx, int nprev, const double* x_stage,
                         const double* y_prev, double* b);

/* Solves A^R y = b (Eq. 3.10) for the last assembled psi^k and tau with
 * FGMRES(restart), modified Gram-Schmidt and right preconditioner P_CH
 * (Sections 4 and 7), zero initial guess.  b, y: 3n doubles on the device.
 * Synchronises the stream to fill *stats (may be NULL).  Returns
 * PFC_ERR_NOT_CONVERGED with the last iterate in y when max_outer is hit. */
pfc_status pfc_stage_solve(pfc_ctx* ctx, const double* b, double* y,
                           pfc_solve_stats* stats);

/* One attempted Ros3Pw step (Eq. 3.6, 3.7, 3.12): assembly at the state,
 * three stage solves, x^{k+1} = x^k + sum m_j y_j and the embedded error
 * estimate err = RMS_j( e_j / (atol + rtol max(|psi^k_j|, |psi^{k+1}_j|)) ) with
 * e = sum (mhat_j - m_j) dpsi_j.  If err <= 1 the step is accepted and state
 * (3n, device, in/out) is overwritten with x^{k+1}; otherwise state is left
 * unchanged.  *tau (in/out) becomes tau * min(5, max(0.2, 0.9 err^(-1/3))),
 * capped at tau_max (and by options.tau_guard); an accepted step that follows a rejected one (on this
 * context) does not grow tau (Hairer-Wanner's rule after a rejection).  stats (may be NULL) receives 3 entries.  One host
 * synchronisation per call. */
pfc_status pfc_step(pfc_ctx* ctx, double* state, double* tau, int* accepted,
                    double* err, pfc_solve_stats* stats);

/* One step of the linearised semi-implicit Euler scheme (Section 3, Eq. 3.3-3.4,
 * PFC2 with K_+ = K): with psi_k from state (3n, device, in/out) and tau_k = tau,
 * assembles A = [[M, -(1+r) M + N(psi_k) + 2 K, K], [tau K, M, 0], [0, K, M]] and
 * b = [(-2 psi_k^3, phi) | M psi_k | 0], solves A x = b with the stage solver
 * (FGMRES(restart) + MGS, P_CH with gamma = 1, zero initial guess) and, when the
 * solve converges, overwrites state with x = [mu | psi | omega]_{k+1}.  On any
 * error state is left unchanged.  Afterwards pfc_apply and pfc_stage_solve use
 * this Euler matrix until the next pfc_assemble or pfc_step.  *stats (may be
 * NULL) receives the solve's statistics.  One host synchronisation per call. */
pfc_status pfc_euler_step(pfc_ctx* ctx, double* state, double tau,
                          pfc_solve_stats* stats);

/* Consistent initial state from psi0 (n doubles, device): solves
 * M omega0 = -K psi0 and M mu0 = (psi0^3, phi) + (1+r) M psi0 - 2 K psi0 - K omega0
 * (the algebraic rows of Eq. 2.4) with float64 Jacobi-PCG to 1e-14 and writes
 * state = [mu0 | psi0 | omega0] (3n, device). */
pfc_status pfc_init_state(pfc_ctx* ctx, const double* psi0, double* state);

/* Operators for checking the path piece by piece (all after pfc_assemble):
 * y = op(x) with op = PFC_OP_M, PFC_OP_K, PFC_OP_A01 (n -> n), PFC_OP_AR (the
 * stage matrix A^R, 3n -> 3n) or PFC_OP_PCH (one application of the
 * preconditioner, 3n -> 3n, with the context's inner precision). */
enum { PFC_OP_M = 0, PFC_OP_K = 1, PFC_OP_A01 = 2, PFC_OP_AR = 3, PFC_OP_PCH = 4 };
pfc_status pfc_apply(pfc_ctx* ctx, int op, const double* x, double* y);

/* One Jacobi-PCG solve (Table 2) A x = b with A = M (which = 0),
 * M + delta K (1) or M + sqrt(delta) K (2), zero start, relative tolerance
 * rtol, in the context's inner precision.  b, x: n doubles on the device.
 * *iterations (may be NULL) receives the iteration count. */
pfc_status pfc_pcg(pfc_ctx* ctx, int which, const double* b, double* x, double rtol,
                   int* iterations);

/* Batched solves of independent instances (not in the paper: many simulations
 * advanced together).  All contexts must live on the same device, share the same
 * CUDA stream and inner precision, and appear once.  One cooperative launch (or
 * one per wave, when there are more instances than co-resident blocks) runs every
 * instance's FGMRES stage solve at once: the grid is split into segments, one per
 * instance, sized by its rows, and each segment runs the solver of
 * pfc_stage_solve with its own barriers and reductions, so an instance's result
 * matches its single-instance solve to the solver tolerance (the block partition,
 * hence the summation order, differs).
 *
 * pfc_batch_stage_solve: y[k] = (A^R_k)^{-1} b[k] for the last pfc_assemble of
 * each context (device pointers, 3n_k doubles each); stats (may be NULL) gets
 * count entries.  Synchronises once.
 *
 * pfc_batch_step: one pfc_step for every instance (states[k]: 3n_k doubles on
 * the device, in/out; taus[k] in/out; accepted, errs (may be NULL) and stats
 * (3 x count, may be NULL) out).  The three stages of all instances are solved by
 * three batched launches; one host synchronisation per call.  The worst status of
 * the instances is returned; every instance's outputs are filled. */
pfc_status pfc_batch_stage_solve(pfc_ctx* const* ctxs, int count, const double* const* b, double* const* y,
                                 pfc_solve_stats* stats);
pfc_status pfc_batch_step(pfc_ctx* const* ctxs, int count, double* const* states, double* taus, int* accepted,
                          double* errs, pfc_solve_stats* stats);

/* A step in three stage launches, for continuous batching (not in the paper: its runs
 * advance one simulation).  A server can then start a newly arrived simulation's
 * step in the same launch that solves the second or third stage of others.
 *
 * pfc_step_begin: assembly at state (3n, device; read here and not kept) for width
 * tau, as in pfc_step; enqueued, no synchronisation.  The context's stage becomes 0.
 *
 * pfc_batch_stage_advance: every context (each after pfc_step_begin, stage 0..2;
 * same device, stream and inner precision; each once) forms its current stage's
 * value x_i and right-hand side b_i^R (Eq. 3.10) and all of them solve their stage
 * systems in one batched persistent launch (more launches when they exceed one
 * co-resident grid); each context's stage then advances by one.  Contexts with
 * options.grid_blocks > 0 keep their own block count and get the same bits as
 * pfc_step.  One host synchronisation per call.  PFC_ERR_INVALID if a context has
 * no begun step or has solved all three stages.
 *
 * pfc_step_finish: after the third stage, the step combination, error estimate,
 * acceptance and next width exactly as pfc_step (same arguments, same state
 * update, stats receives 3 entries); the context's stage becomes -1.
 *
 * pfc_step_stage: the context's stage: -1 no begun step, 0..2 the next stage to
 * solve, 3 ready for pfc_step_finish.  Every other step, assembly or solve call
 * abandons a begun step. */
pfc_status pfc_step_begin(pfc_ctx* ctx, const double* state, double tau);
pfc_status pfc_batch_stage_advance(pfc_ctx* const* ctxs, int count);
pfc_status pfc_step_finish(pfc_ctx* ctx, double* state, double* tau, int* accepted, double* err,
                           pfc_solve_stats* stats);
int pfc_step_stage(const pfc_ctx* ctx);

/* Failure-detection self-test: launches a PCG whose grid barriers wait for one
 * block more than the grid holds, so every wait runs out after limit_seconds
 * (0 < limit <= 10).  The kernel sets its timeout bit and returns; the context
 * stays usable.  Returns PFC_ERR_TIMEOUT when the bounded wait works.  (Not a
 * step of the paper's method: it checks the persistent kernel's bounded waits.) */
pfc_status pfc_selftest_barrier_timeout(pfc_ctx* ctx, double limit_seconds);

/* Accounting for benchmarks.  pfc_set_timing(ctx, 1) makes every later
 * persistent-solver launch record CUDA events on the context stream around
 * itself; the elapsed times are summed at the next synchronising call.
 * pfc_counters reports the number of kernels the context has launched, the
 * number of persistent-solver launches and the summed solver time (ms).
 * Either output pointer may be NULL. */
pfc_status pfc_set_timing(pfc_ctx* ctx, int enable);
pfc_status pfc_counters(const pfc_ctx* ctx, long long* kernel_launches, long long* solver_launches,
                        double* solver_ms);

/* Host-only inspection of the mesh/pattern builder (no GPU needed):
 * out4 = {n, nnz of one block, stored SELL slots, elements}. */
pfc_status pfc_host_pattern(int dim, int side, double length, int64_t* out4);

/* Row-block partition of one instance over nparts devices (host only, no GPU).
 * The paper's parallel runs distribute the rows of the stage system over MPI
 * processes in contiguous blocks, with a halo exchange per matrix-vector product
 * and a global sum per inner product (PETSc, Section 7).  This is the plan such a
 * multi-device solve uses here: each field's lexicographic rows (same cut in
 * mu, psi and omega) are split into nparts strips of whole lattice lines (2D) or
 * planes (3D), balanced by nonzeros; a strip's columns reach at most `degree`
 * lines beyond it, so it exchanges ghost values with its two neighbours only.
 * row_begin (nparts + 1): first row of each part and n; halo (2 nparts): ghost
 * rows below and above part k (in [2k], [2k + 1]); part_nnz (nparts): nonzeros of
 * one block in part k.  PFC_ERR_INVALID for bad sizes or when a part would hold
 * fewer than `degree` lines.  This build runs one device per instance; the plan is
 * exercised by a multi-process CPU test of the partitioned solve. */
pfc_status pfc_host_partition(int dim, int side, double length, int degree, int nparts, int64_t* row_begin,
                              int64_t* halo, int64_t* part_nnz);

/* Host-only inspection of the P2 cell-major order (no GPU needed; options.cells; dim 2 or 3):
 * out4 = {row classes (distinct row stencils; the first four are the interior
 * stencils of the dof types, the fifth is the empty stencil of padding rows),
 * stencil entries over all row classes, cell classes (distinct tuples of a 2 x 2
 * cell's rows' classes) if the interior stencils extracted from the assembled
 * pattern are the couplings the cell kernels hard-code (cell2d.h, cell3d.h) and every other
 * row couples to a subset of them, else 0 (the cell kernels then stay off), rows that
 * hold a dof}.  The stencils are those of the P2 matrices of Section 3 on this
 * structured mesh. */
pfc_status pfc_host_cells(int dim, int side, double length, int64_t* out4);

/* 1 if the context's float32/float16 inner solves run the cell kernels
 * (options.cells with 2D P2 structured stencils, the Chronopoulos-Gear form and room
 * in shared memory), else 0 (also for NULL or float64 contexts).  Host only. */
int pfc_cell_kernels(const pfc_ctx* ctx);

/* Host-only inspection of the structured stencils (no GPU needed):
 * out3 = {rows that use the stencil, nonzeros of the rows that keep their
 * assembled values, stencil entries over all dof types}. */
pfc_status pfc_host_stencil(int dim, int side, double length, int64_t* out3);

/* Step combination and embedded error estimate for callers that cannot
 * allocate device memory: code inside a CUDA stream capture, a loop that must not
 * touch the allocator once running, or a guest whose host application owns all
 * device memory cannot create a context, but can combine stage increments it
 * already holds.  (The paper has no counterpart: this is a packaging of the
 * step combination of pfc_step.)
 *   state_new = state + sum_j m_j y_j          (3n doubles, device, written)
 *   *err      = RMS over the psi block [n, 2n) of e / (atol + rtol max(|psi|, |psi_new|)),
 *               e = sum_j (mhat_j - m_j) y_j   (1 double, device, written)
 * state: 3n doubles [mu | psi | omega]; y: the three stage increments back to
 * back (3 x 3n doubles); all device pointers; m, mhat from Table 1.  Work is
 * enqueued on cuda_stream (NULL = legacy default stream); nothing synchronises.
 * Allocates nothing: the only working memory is an 8 KiB array of per-block
 * partial sums in static device memory of the library, which every GPU that loads
 * the library keeps until the process exits.  The first call on a device looks
 * up that array's device address (with the device current); make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents; each call overwrites the partials it reads, so nothing needs
 * clearing, but two calls whose kernels overlap on the GPU (different streams, or
 * several host threads) race on it and must be serialised by the caller.
 * Returns PFC_ERR_INVALID for n < 1, n > 715740501 (= (2^31 - 1 - 2^18) / 3: the
 * kernel's 32-bit index, stepping by 2^18, must not pass 2^31 - 1 on its way past
 * 3n), null pointers or bad tolerances, PFC_ERR_CUDA if a launch fails. */
pfc_status pfc_step_combine_static(int64_t n, const double* state, const double* y, double atol, double rtol,
                                   double* state_new, double* err, void* cuda_stream);

/* Text of the most recent error of ctx ("" if none; static text for NULL). */
const char* pfc_last_error(const pfc_ctx* ctx);

/* Name of a status code. */
const char* pfc_status_string(int status);

/* Frees every device buffer of ctx.  NULL is ignored. */
void pfc_destroy(pfc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PFC_H */
