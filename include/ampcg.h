/*
 * ampcg.h -- C ABI of the B300 (sm_103a) adaptive mixed-precision,
 * dynamically scaled preconditioned conjugate gradient library.
 *
 * Method: Guo, de Sturler, Warburton, "An Adaptive Mixed-Precision and
 * Dynamically Scaled Preconditioned Conjugate Gradient Algorithm"
 * (arXiv 2505.04155).  Section and equation names below refer to that paper.
 *
 * Conventions for every entry point:
 *   - Return codes only: no exception crosses the ABI, the library never
 *     aborts and never traps on the device.  After a non-OK status,
 *     ampcg_last_error() holds a one-line description (per thread).
 *   - The caller owns every array it passes.  ampcg_create_csr copies the
 *     matrix into library-owned device memory; the caller may free its arrays
 *     as soon as the call returns.
 *   - "device or host" pointers: the library asks the CUDA runtime which kind
 *     a pointer is and copies host data to/from the device itself.
 *   - All work of a context is ordered on the CUDA stream given at creation
 *     (NULL: the library creates its own non-blocking stream).  Calls that
 *     return results to the host synchronise that stream before returning.
 *   - One context must not be used from two threads at the same time.
 */
#ifndef AMPCG_H
#define AMPCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque solver context: one SPD matrix with its preconditioner, its
 * precision copies and its device work buffers. */
typedef struct ampcg_ctx* ampcg_t;

/* Floating-point formats.  Ordered from high to low precision; the "min" of
 * two precisions in Eq. (precision_selector) is the larger code. */
typedef enum { AMPCG_FP64 = 0, AMPCG_FP32 = 1, AMPCG_FP16 = 2 } ampcg_prec;

typedef enum {
  AMPCG_OK = 0,                /* converged (updated residual <= tol*||b||) */
  AMPCG_NOT_CONVERGED = 1,     /* maxit reached; x and histories are filled */
  AMPCG_ERR_INVALID_ARG = -1,  /* bad size, pointer, policy or CSR structure */
  AMPCG_ERR_NOT_SPD = -2,      /* create-time evidence: a diagonal entry <= 0 */
  AMPCG_ERR_BREAKDOWN = -3,    /* rho_k <= 0 or gamma_k <= 0 in Alg. 3 */
  AMPCG_ERR_NONFINITE = -4,    /* NaN/Inf in b, x0 or a recurrence scalar */
  AMPCG_ERR_CUDA = -5,         /* a CUDA runtime call failed */
  AMPCG_ERR_OOM = -6,          /* device allocation failed */
  AMPCG_ERR_TIMEOUT = -7,      /* a bounded device wait ran out */
  AMPCG_ERR_NO_DEVICE = -8,    /* no CUDA device is visible */
  AMPCG_ERR_UNSUPPORTED = -9   /* valid request the library does not support */
} ampcg_status;

/* Preconditioner M (Alg. 3 applies M^-1 to the scaled residual). */
typedef enum { AMPCG_M_NONE = 0, AMPCG_M_JACOBI = 1, AMPCG_M_CHEBYSHEV = 2 } ampcg_m_type;

/* Jacobi: M = diag(A).  Chebyshev: M^-1 = D^-1/2 P(Ahat) D^-1/2 with
 * Ahat = D^-1/2 A D^-1/2 and P the polynomial of `degree` steps of the
 * Chebyshev iteration for Ahat (Saad, Alg. 12.1) from zero on [lmin, lmax]
 * (degree - 1 products with the copy of Ahat in u_z per application). */
typedef struct {
  int type;        /* ampcg_m_type */
  int degree;      /* Chebyshev: number of Chebyshev steps m, 1..64 */
  double lmin;     /* Chebyshev: interval [lmin, lmax] for Ahat.  lmax <= 0:  */
  double lmax;     /*   lmax = Gershgorin bound max_i sum_j |ahat_ij| (an upper */
                   /*   bound of the spectrum, so M stays SPD); lmin <= 0:      */
                   /*   lmin = lmax / 30                                        */
} ampcg_precond_spec;

/* Criterion for the u_r switch (Sec. 4.1). */
typedef enum {
  AMPCG_CRIT_WINDOW = 0,  /* delay-window indicator, Eq. (eta_k), d and C */
  AMPCG_CRIT_LINEAR = 1,  /* linear-convergence indicator, Eq. (linear criterion), ell and C */
  AMPCG_CRIT_FIXED = 2    /* no selector: (u_z, u_r) = (fixed_uz, fixed_ur); FP64/FP64 = PCG */
} ampcg_criterion;

/* Dynamic scaling omega_k of y_k = omega_k r_k (Alg. 2, Alg. 3). */
typedef enum {
  AMPCG_SCALE_NONE = 0,      /* omega = 1 (plain PCG) */
  AMPCG_SCALE_L2 = 1,        /* omega = 1/||r_k||, as printed in Alg. 3 */
  AMPCG_SCALE_LINF_POW2 = 2, /* omega = 2^-ceil(log2 max|r_k|): exact, max|y| in (0.5, 1].
                                The persistent iteration kernel forms z_{k+1} and rho_{k+1} in
                                its update step with the exponent of max|r_k| and keeps them
                                when max|r_{k+1}| has that exponent (then they are the ones
                                this omega gives, bit for bit); otherwise the iteration forms
                                them again (see ampcg_tune). */
  AMPCG_SCALE_LINF_POW2_LAG = 3 /* omega_k = 2^-ceil(log2 max|r_{k-1}|) (k >= 1; omega_0 from r_0):
                                 the previous iteration's power of two, a lagged factor as
                                 Sec. 3.3 allows; if rho_k comes out non-finite (y_k overflowed
                                 u_z), y_k, z_k and rho_k are formed again with
                                 2^-ceil(log2 max|r_k|).  Known before delta_{k+1} is reduced,
                                 so the persistent iteration kernel forms z_{k+1} and rho_{k+1}
                                 in its update step (three grid barriers per iteration instead
                                 of four).  Not with the Chebyshev preconditioner
                                 (AMPCG_ERR_UNSUPPORTED). */
} ampcg_scale;

typedef struct {
  int u0;             /* initial (maximum) u_z precision, ampcg_prec */
  int criterion;      /* ampcg_criterion */
  int d;              /* window delay d of Eq. (eta_k); paper: 10; 0..62 */
  int ell;            /* rate window ell of Eq. (linear criterion); paper: 5; 1..63 */
  double C;           /* Assumption 1 constant; paper: 1 */
  double tau_zs;      /* nu_k threshold for u_z -> FP32; paper: 1e-4 */
  double tau_zh;      /* nu_k threshold for u_z -> FP16; paper: 1e-6 */
  int scale;          /* ampcg_scale */
  int latch;          /* 1: a precision never rises again within a solve */
  int verify_refresh; /* >0: after convergence verify b - A x in FP64 and, if
                         it exceeds tol*||b||, replace r and continue; at most
                         this many times.  0: stop on the updated residual. */
  int fixed_uz;       /* FIXED criterion only */
  int fixed_ur;       /* FIXED criterion only: AMPCG_FP64 or AMPCG_FP32 */
  int graph_chunk;    /* iterations per chunk of the device-side loop: per launch of the
                         persistent iteration kernel (Jacobi or none), or per repeat of
                         the kernel sequence (>= 1; 0 = automatic: 256 for the
                         persistent kernel, 16 for the sequence) */
} ampcg_policy;

typedef struct {
  int iters;              /* iterations performed (Alg. 3 loop trips) */
  int converged;          /* 1 if the updated residual met tol*||b|| */
  int refreshes;          /* true-residual replacements performed */
  int status;             /* ampcg_status of the solve */
  double true_relres;     /* ||b - A x||_2 / ||b||_2 recomputed in FP64 at exit */
  double updated_relres;  /* delta_iters / ||b|| */
  int switch_iter[3];     /* first iteration with u_z = FP32, u_z = FP16, u_r = FP32
                             reached by a change of precision; -1 if none */
  double seconds;         /* wall time of the call */
  double* relres_hist;    /* caller-owned host array, length >= maxit + 1, or NULL:
                             receives delta_k / ||b||, k = 0..iters */
  uint8_t* prec_hist;     /* caller-owned host array, length >= maxit, or NULL:
                             receives (u_z << 4) | u_r used at iteration k */
  int64_t kernel_launches; /* library kernels launched by the call (graph nodes included) */
} ampcg_result;

/* Fills *p with the paper's defaults (d = 10, C = 1, ell = 5, tau_zs = 1e-4,
 * tau_zh = 1e-6, Sec. 5) for AMP-PCG(FP16) with the linear criterion,
 * LINF_POW2 scaling, latching on, verify_refresh = 0. */
void ampcg_policy_default(ampcg_policy* p);

/* Creates a context for the SPD matrix A given in CSR form (Sec. 2: A is
 * SPD; Alg. 3 REQUIRE: A, M).  n rows; rowptr[n+1] (int32, rowptr[0] = 0,
 * nondecreasing, rowptr[n] = nnz); colind[nnz] (int32, in [0, n), strictly
 * increasing within each row); vals[nnz] FP64.  Arrays may be host or device
 * pointers.  The library validates the structure and the diagonal
 * (AMPCG_ERR_INVALID_ARG, AMPCG_ERR_NOT_SPD), then builds on the device the
 * FP64 and FP32 copies of A in its internal sliced layout, the Jacobi inverse
 * diagonal in FP64/FP32/FP16 and, for Chebyshev, the FP64/FP32/FP16 copies of
 * D^-1/2 A D^-1/2 and of D^-1/2.  cuda_stream: a cudaStream_t or NULL.  On success *out
 * owns device memory until ampcg_destroy. */
ampcg_status ampcg_create_csr(ampcg_t* out, int64_t n, int64_t nnz, const int32_t* rowptr,
                              const int32_t* colind, const double* vals,
                              const ampcg_precond_spec* M, void* cuda_stream);

/* Creates a context from block CSR: nb block rows of bs x bs blocks (1 <= bs
 * <= 16), browptr[nb+1] (0 .. nnzb), bcolind[nnzb] (block columns in
 * [0, nb), strictly increasing within a block row), bvals[nnzb * bs * bs]
 * (each block row-major).  The blocks are expanded on the device into the
 * scalar matrix of n = nb * bs rows (row I*bs + r takes row r of every block
 * of block row I), which then goes through the same validation and
 * preparation as ampcg_create_csr; all other calls see the scalar system
 * (vectors of length nb * bs, dL/dA in the expanded CSR order).  With bs = 3
 * and rows wider than 8 entries the context also keeps a block-row layout
 * (one block column index and 9 values per block, the values also as
 * D^-1/2 A D^-1/2 for Chebyshev), which the Chebyshev steps and the
 * SpMV of the kernel sequence use: one thread per block row gathers each
 * block's 3 operands once for its 3 rows, in the same order of operations
 * as the scalar layout (bitwise the same results). */
ampcg_status ampcg_create_bsr(ampcg_t* out, int64_t nb, int bs, int64_t nnzb, const int32_t* browptr,
                              const int32_t* bcolind, const double* bvals,
                              const ampcg_precond_spec* M, void* cuda_stream);

/* The Chebyshev interval in use (after automatic choice).  Returns
 * AMPCG_ERR_INVALID_ARG for other preconditioners. */
ampcg_status ampcg_precond_interval(ampcg_t ctx, double* lmin, double* lmax);

/* Releases every resource of the context (NULL is ignored). */
void ampcg_destroy(ampcg_t ctx);

/* Replaces the matrix values, keeping the sparsity pattern given at creation:
 * vals[nnz] FP64 in the same CSR order (host or device).  Rebuilds the FP64
 * and FP32 copies and the Jacobi inverse diagonal on the device.  Returns
 * AMPCG_ERR_NONFINITE / AMPCG_ERR_NOT_SPD if a value is not finite or a
 * diagonal entry is not positive (the context then holds the new values and
 * must not be solved with).  Synchronises the context's stream. */
ampcg_status ampcg_update_values(ampcg_t ctx, const double* vals);

/* Solves A x = b with AMP-PCG (Alg. 3; Alg. 1 and Alg. 2 under the FIXED
 * criterion).  b[n] FP64 (device or host); x[n] FP64 (device or host), in:
 * x_0, out: the final iterate.  tol > 0: stop when ||r_{k+1}|| <= tol ||b||
 * (the stopping test of Alg. 3).  maxit >= 0.  policy NULL = ampcg_policy_default.
 * res (may be NULL) receives counts, final residuals, switch points and, when
 * its history pointers are set, the per-iteration residual and precision
 * histories.  Returns the solve's status (AMPCG_OK, AMPCG_NOT_CONVERGED,
 * AMPCG_ERR_BREAKDOWN, AMPCG_ERR_NONFINITE) or an error (AMPCG_ERR_TIMEOUT:
 * a bounded grid-barrier wait of the persistent iteration kernel ran out, a
 * block never arrived; the solve stops instead of hanging); x holds the last
 * iterate in every non-error case.  Synchronises the context's stream. */
ampcg_status ampcg_solve(ampcg_t ctx, const double* b, double* x, double tol, int maxit,
                         const ampcg_policy* policy, ampcg_result* res);

/* Solves nsys independent systems (distinct contexts, each with its own
 * b[i] and in/out x[i], host or device, n_i doubles) with the same tol, maxit
 * and policy, after all work already queued on the contexts' streams and
 * before any work queued there later.  Each system stops on its own test.
 *   - Systems of at most 131072 rows with Jacobi or no preconditioner run in
 *     one persistent launch: a block of 1024 threads solves one system at a
 *     time (block-level reductions, state in shared memory), taking systems
 *     largest first.  Iterates agree with ampcg_solve to rounding (the
 *     reduction order differs); a system's result does not depend on the
 *     rest of the batch.
 *   - Other systems run ampcg_solve's device loop on library streams (up to
 *     16 at a time): bitwise equal to ampcg_solve.
 * results[i] (may be NULL) as in ampcg_solve; the persistent launches are
 * counted in kernel_launches of the first system that used them.  Returns
 * AMPCG_OK if every system converged, AMPCG_NOT_CONVERGED if some reached
 * maxit, else the first failing system's status (ampcg_last_error names it).
 * Synchronous.  Not from the paper. */
ampcg_status ampcg_solve_batched(int nsys, ampcg_t const* systems, const double* const* b,
                                 double* const* x, double tol, int maxit,
                                 const ampcg_policy* policy, ampcg_result* results);

/* Per-kernel device time of one solve, split by the precision pair of the
 * iteration, as the paper reports per-kernel time for each phase of
 * AMP-PCG (Sec. 5.5).  Index [kernel][phase]: kernel 0 = scale+precondition
 * +rho+beta (with Jacobi or no preconditioner also the search direction),
 * 1 = search direction (Chebyshev), 2 = SpMV+gamma+alpha, 3 = x/r
 * update+norm+stopping test+selector (the steps of Alg. 3); phase =
 * 2*u_z + u_r (u_z in {FP64, FP32, FP16}, u_r in {FP64, FP32}).  Where the
 * whole iteration is one launch of the persistent iteration kernel (Jacobi
 * or none, slices at most 8 entries wide), it is timed in slot 0, one
 * iteration per launch, and slots 1-3 stay empty. */
typedef struct {
  double ms[4][6];     /* summed CUDA-event durations */
  int launches[4][6];  /* launches that did work */
  double total_ms;     /* device time from the first to the last launch */
} ampcg_kernel_times;

/* Same as ampcg_solve, computing the same iterates bit for bit, but the
 * iteration kernels are launched one by one (no graph; the persistent kernel
 * with one iteration per launch) with a CUDA event pair around each launch,
 * and their durations are returned in *kt.  Slower than
 * ampcg_solve by the launch overhead; meant for measurement. */
ampcg_status ampcg_solve_timed(ampcg_t ctx, const double* b, double* x, double tol, int maxit,
                               const ampcg_policy* policy, ampcg_result* res,
                               ampcg_kernel_times* kt);

/* Adjoint of the solve x = A^-1 b for a scalar loss L(x): given x (the
 * forward solution) and g = dL/dx, solves A lambda = g (A is symmetric, Sec. 2)
 * with the same AMP-PCG and policy, from lambda_0 = 0, so lambda = dL/db; and
 * if dLdA_vals is not NULL writes dL/da_ij = -lambda_i x_j for every stored
 * entry, in the CSR order given at creation (nnz values).  x, dLdx, lambda,
 * dLdA_vals: FP64, host or device.  Status as ampcg_solve.  The paper has no
 * adjoint; this is the standard adjoint identity dL/dA = -lambda x^T
 * restricted to the pattern.  Synchronises the context's stream. */
ampcg_status ampcg_adjoint(ampcg_t ctx, const double* x, const double* dLdx, double tol, int maxit,
                           const ampcg_policy* policy, double* lambda, double* dLdA_vals,
                           ampcg_result* res);

/* Log-coefficient field on the matrix graph.  For a pattern whose stored
 * off-diagonals are the faces (i, j) of a node graph, sets
 *   a_ij = -exp((theta_i + theta_j)/2),
 *   a_ii = sum_{j != i} exp((theta_i + theta_j)/2) + nbound_i exp(theta_i)
 * (a 7-point diffusion operator with face coefficients exp of the mean log
 * coefficient, nbound_i = number of Dirichlet boundary faces of node i), and
 * rebuilds the value copies and the Jacobi diagonal.  theta[n] FP64,
 * nbound[n] int32, host or device.  Every row must store its diagonal
 * (AMPCG_ERR_INVALID_ARG otherwise).  Not from the paper (coefficient-field
 * workloads for the adjoint).  Synchronises the context's stream. */
ampcg_status ampcg_assemble_log_coeff(ampcg_t ctx, const double* theta, const int32_t* nbound);

/* Chain rule to the log-coefficient field for the current values: with x
 * the forward solution and lambda the adjoint solution (ampcg_adjoint),
 * writes dL/dtheta_i = sum_{j != i} -(lambda_i - lambda_j)(x_i - x_j)(-a_ij)/2
 * - lambda_i x_i (sum_j a_ij), which is dL/da_ij = -lambda_i x_j pushed
 * through ampcg_assemble_log_coeff's formula.  FP64 arrays of length n, host
 * or device.  Synchronises the context's stream. */
ampcg_status ampcg_grad_log_coeff(ampcg_t ctx, const double* x, const double* lambda,
                                  double* dLdtheta);

/* --- Single steps of the iteration, on device arrays of length n ---------- */

/* q = A p in precision `prec` (the matrix product of Alg. 3): the FP64 or FP32 copy of A,
 * one fused multiply-add per stored entry in ascending column order,
 * accumulated in `prec`.  p and q are device arrays of doubles (FP64) or
 * floats (FP32).  Asynchronous on the context's stream. */
ampcg_status ampcg_spmv(ampcg_t ctx, int prec, const void* p, void* q);

/* z = M^-1 y with y = round_uz(omega * r computed in ur) (the scaling and preconditioning of Alg. 3).
 * r: device array in precision ur (double or float); z: device array in
 * precision uz (double, float or IEEE half as uint16).  omega: the scale
 * factor.  Asynchronous on the context's stream. */
ampcg_status ampcg_precond_apply(ampcg_t ctx, int uz, int ur, double omega, const void* r,
                                 void* z);

/* The matrix product of Alg. 3 as the persistent iteration kernel computes
 * it: q = A p with A's copy in u_r (FP64 or FP32 values, one fma per stored
 * entry in ascending column order, accumulated in u_r) and p stored in u_z
 * (double, float or IEEE half as uint16, widened exactly, or rounded to
 * binary32 when u_z = FP64 and u_r = FP32), launched with that kernel's grid,
 * shared-memory stages and per-warp slice runs, so the code path under test
 * is the solve's own.  p: device array of n values in u_z; q: device array of
 * n values in u_r.  gamma (host, may be NULL) receives q^T p accumulated as
 * the iteration kernel does (per-block partials summed in block order).
 * AMPCG_ERR_UNSUPPORTED for contexts that do not run that kernel (Chebyshev
 * or slices wider than 8 entries).  Synchronises the context's stream. */
ampcg_status ampcg_spmv_loop_step(ampcg_t ctx, int uz, int ur, const void* p, void* q, double* gamma);

/* q = A p with the block-row layout of a context created from 3 x 3 block
 * CSR (ampcg_layout.block3 = 1): the FP64 or FP32 values, one fma per stored
 * entry in ascending column order per row, accumulated in `prec` -- the same
 * result as ampcg_spmv on the expanded matrix.  p, q: device arrays of n
 * values in `prec`.  AMPCG_ERR_UNSUPPORTED without the block layout.
 * Asynchronous on the context's stream. */
ampcg_status ampcg_spmv_block(ampcg_t ctx, int prec, const void* p, void* q);

/* r = b - A x in FP64 (the initial residual of Alg. 3): per row, an FP64 fused multiply-add
 * chain over the stored entries in ascending column order, subtracted from
 * b.  Device arrays of doubles.  Asynchronous on the context's stream. */
ampcg_status ampcg_residual(ampcg_t ctx, const double* b, const double* x, double* r);

/* Runs the device's precision selector (Eq. (precision_selector) with the
 * indicator chosen by policy->criterion, latching as in the policy) over a
 * given residual-norm sequence delta[0..m] (host array), as the solver
 * would at iterations k = 0..m; writes (u_z << 4) | u_r for each k into
 * out[m+1] (host).  nb = ||b||, tol as in ampcg_solve.  0 <= m < 2^28
 * (AMPCG_ERR_INVALID_ARG otherwise, checked before any CUDA call).
 * Synchronous; allocates its device scratch per call. */
ampcg_status ampcg_selector_trace(const ampcg_policy* policy, const double* delta, int m,
                                  double nb, double tol, uint8_t* out);

/* The same selector replay as ampcg_selector_trace, with the same arguments
 * and results, but it allocates no device memory: its device scratch (a state
 * block and three arrays of m+1 entries) lives in one static array compiled
 * into the library, about 650 KB, which every GPU that loads the library
 * holds until the process exits.  It is for callers that must not call
 * cudaMalloc, for example code that runs while a caching allocator has
 * reserved the device's free memory for itself, or latency-critical loops
 * where cudaMalloc's implicit device synchronisation is not acceptable.
 *   - m + 1 must be at most 65536; larger m is rejected with
 *     AMPCG_ERR_INVALID_ARG and nothing is run.
 *   - The first call in a device's context (with that device current)
 *     looks up the array's device address and caches it with the context's
 *     identity; a call in a later context of the device (after a reset of
 *     its primary context) looks it up again.  Make the first call on each
 *     device, and the first after a reset, before any stream capture.
 *   - m + 1 is checked against the limit before any CUDA call.
 *   - All calls share the one array: calls that overlap on the GPU (for
 *     example from two host threads) race and must be serialised by the
 *     caller.  Each call writes everything it reads before reading it.
 *   - Synchronous; uses the legacy default stream, like ampcg_selector_trace.
 * The paper has no counterpart to this entry point. */
ampcg_status ampcg_selector_trace_noalloc(const ampcg_policy* policy, const double* delta, int m,
                                          double nb, double tol, uint8_t* out);

/* Failure detection without a GPU fault (not from the paper).  Runs one grid
 * barrier of the kind the persistent iteration kernel uses (every block
 * publishes a partial, takes a ticket and polls the ticket counter with at
 * most `spin_limit` polls per polling warp, then all blocks sum the partials)
 * in a cooperative launch of `nblocks` blocks, 2 <= nblocks <= 64,
 * 1 <= spin_limit <= 2^21 (about a second).  absent_block in [0, nblocks):
 * that block returns without arriving, so the other blocks' waits run out;
 * -1: every block arrives.  Returns AMPCG_OK when every arriving block
 * passed the barrier with the correct grid sum; AMPCG_ERR_TIMEOUT when a
 * wait ran out -- the status ampcg_solve returns when a barrier wait of its
 * iteration kernel runs out; AMPCG_ERR_INVALID_ARG for bad arguments
 * (checked before any CUDA call).  Allocates a few bytes of device memory;
 * synchronous on the legacy default stream. */
ampcg_status ampcg_barrier_check(int nblocks, int absent_block, long long spin_limit);

/* Autotuning of the persistent iteration kernel (Jacobi or no
 * preconditioner, slices at most 8 wide; not from the paper).  For each
 * precision pair ph = 2 u_z + u_r the kernel runs either the four-barrier
 * iteration (scaling and preconditioning in their own step) or the
 * three-barrier one (z_{k+1}, rho_{k+1} formed in the update step and reduced
 * with delta_{k+1}).  The three-barrier form needs omega_{k+1} before
 * delta_{k+1} is reduced: AMPCG_SCALE_NONE and AMPCG_SCALE_LINF_POW2_LAG know
 * it; under AMPCG_SCALE_LINF_POW2 the update step forms z_{k+1} with the
 * exponent of max|r_k| and keeps it when max|r_{k+1}| has the same exponent
 * (then omega_{k+1} is that power of two and z_{k+1} is bit for bit the one
 * the four-barrier form computes), else the iteration forms it again in its
 * own step.  AMPCG_SCALE_L2 has the four-barrier form only.  Both forms
 * compute Alg. 3; their inner products differ only in summation order.
 * Without tuning the three-barrier form is used. */
typedef struct {
  int fused[6];        /* per pair: 1 three-barrier form, 0 four-barrier, -1 automatic */
  double us_plain[6];  /* measured device time per iteration, four-barrier form (0: not timed) */
  double us_fused[6];  /* the same, three-barrier form */
  int iters;           /* iterations timed per form and pair */
  int cached;          /* 1: taken from this process's cache of an equal matrix shape */
  int reserved;        /* pairs measured (bit mask) */
  int pad;
} ampcg_tuning;

/* Measures, on the context's own matrix and under the scale mode `scale`
 * (AMPCG_SCALE_NONE, AMPCG_SCALE_LINF_POW2_LAG or AMPCG_SCALE_LINF_POW2, the
 * modes with two forms, tuned separately; AMPCG_ERR_INVALID_ARG for
 * AMPCG_SCALE_L2), `iters` (1..10000) iterations of both
 * forms for every pair in the bit mask `pairs` (bit ph; 0 = all six), as the
 * difference of two fixed-pair solves of iters and 2 iters iterations (CUDA
 * events, the best of three timings of each; fixed costs cancel; where the
 * difference is not positive, as on a small system whose fixed costs swamp
 * it, both forms are compared on their 2 iters solves, per iteration), keeps
 * the faster form per pair in the context
 * for later solves under that scale mode, and fills *out.  Results are cached
 * per matrix shape (rows, entries, layout, preconditioner, device) and scale
 * mode within the process: a later call for an equal shape reuses them
 * (out->cached = 1).  Contexts without the persistent kernel get fused[] = -1
 * and AMPCG_OK; so does a pair whose timing solve (right-hand side of ones,
 * x_0 = 0) breaks down or stops early on this system (for example binary16
 * z without scaling).  Allocates two vectors of n doubles; synchronous. */
ampcg_status ampcg_tune(ampcg_t ctx, int scale, int iters, int pairs, ampcg_tuning* out);

/* Applies the forms of t->fused[] (-1, 0 or 1 per pair) for solves under the
 * scale mode `scale` (as ampcg_tune; for example a tuning saved from an
 * earlier process); other fields are ignored. */
ampcg_status ampcg_set_tuning(ampcg_t ctx, int scale, const ampcg_tuning* t);

/* Autotuning of ampcg_solve_batched's persistent kernel (not from the paper):
 * its block size, 1024 threads (one system per SM at a time) or 512 (two per
 * SM, each with half the threads).  Runs the batch twice per candidate (the
 * first a warm-up) with `iters` (1..10000) iterations per system under
 * `policy` (NULL: default) on right-hand sides of ones, wall-clock timed, and
 * stores the faster size in every system's context (the batch uses the size
 * stored in its first eligible system).  Allocates 2 sum(n_i) doubles;
 * synchronous. */
typedef struct {
  int block[2];      /* candidates: 1024, 512 */
  double ms[2];      /* measured wall time of the batch per candidate */
  int chosen;        /* the size stored */
  int iters;
} ampcg_batch_tuning;
ampcg_status ampcg_tune_batched(int nsys, ampcg_t const* systems, const ampcg_policy* policy, int iters,
                                ampcg_batch_tuning* out);

/* Sets the batched kernel's block size for batches led by these contexts:
 * 0 (default, 1024), 1024 or 512. */
ampcg_status ampcg_set_batch_block(int nsys, ampcg_t const* systems, int block);

/* Number of rows of the context's matrix, or -1 for NULL. */
int64_t ampcg_rows(ampcg_t ctx);

/* Storage statistics of the context's matrix in the sliced layout (slices of
 * 32 rows, entry j of a slice's rows stored together; column offsets in int16
 * when they fit).  A slice whose rows all have their entries at one set of
 * offsets is stored with that set (added entries hold exact zeros) and the
 * SpMV reads its 8 offsets once instead of per entry: stored_uniform counts
 * the entries of such slices.  For byte models; not from the paper.  Returns
 * AMPCG_ERR_INVALID_ARG for NULL arguments; synchronises the context's
 * stream. */
typedef struct {
  int64_t n;               /* rows */
  int64_t nslices;         /* slices of 32 rows */
  int64_t stored;          /* stored entries (32 x width summed over slices) */
  int64_t stored_uniform;  /* of these, in slices with uniform offsets */
  int32_t maxw;            /* largest slice width */
  int32_t idx16;           /* 1: int16 column offsets, 0: int32 columns */
  int32_t stream_hint;     /* 1: matrix loads carry an L2 evict-first hint */
  int32_t block3;          /* 1: created from 3 x 3 block CSR; the Chebyshev steps and the
                              SpMV of the kernel sequence use the block-row layout (one block
                              column and 9 values per block, one thread per block row) */
} ampcg_layout;
ampcg_status ampcg_layout_stats(ampcg_t ctx, ampcg_layout* out);

/* Static strings: a status name, and the last error of this thread. */
const char* ampcg_status_string(int status);
const char* ampcg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AMPCG_H */
