/*
 * esdcg — deflated / subspace-corrected ICCG for a sequence of SPD systems with one matrix,
 * the auxiliary matrix W built from error vectors sampled during an earlier solve
 * (arXiv 2203.08498). One GPU (sm_103a); every numerical step runs in this library's CUDA
 * kernels.
 *
 * Conventions for every entry point:
 *   - Return value: ESD_OK (0) or a negative ESD_ERR_* code; esd_last_error() then returns
 *     a message (library-owned, valid until the next failing call on the same thread).
 *   - Vectors are arrays of n doubles. "Device or host" arguments may point to device memory
 *     or to host memory (pinned or pageable); host data is staged through library buffers.
 *   - The library never frees, keeps or aliases caller memory beyond the call: inputs are
 *     copied in, outputs copied out.
 *   - All work is ordered on the stream given to esd_create_matrix. Calls that return values
 *     to the host (iteration counts, norms, estimates) synchronise that stream.
 *   - Handles are not thread-safe; use one handle per host thread or serialise calls.
 */
#ifndef ESDCG_H
#define ESDCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum esd_status {
  ESD_OK = 0,
  ESD_ERR_INVALID = -1,   /* bad argument, malformed CSR or colouring */
  ESD_ERR_NOT_SPD = -2,   /* IC(0) pivot <= 0 after every allowed diagonal shift */
  ESD_ERR_BREAKDOWN = -3, /* (p, Ap) <= 0 or (r, z) <= 0 or NaN during a solve */
  ESD_ERR_MAXIT = -4,     /* tolerance not reached in maxit iterations (x holds the last iterate) */
  ESD_ERR_STATE = -5,     /* call not valid in the current state (e.g. deflation without W) */
  ESD_ERR_RANK = -6,      /* the sampled error vectors have rank 0 */
  ESD_ERR_CHOL_E = -7,    /* E = W^T A W is not numerically positive definite */
  ESD_ERR_CUDA = -8,      /* a CUDA runtime call failed */
  ESD_ERR_NOMEM = -9,     /* device allocation failed */
  ESD_ERR_INTERNAL = -10  /* an internal guard stopped the device loop (a library defect) */
};

enum esd_mode {
  ESD_PLAIN = 0,                  /* PCG with M^{-1} */
  ESD_DEFLATION = 1,              /* deflated PCG, Algorithm "Deflated PCG" */
  ESD_SUBSPACE_CORRECTION = 2     /* PCG with M_sc^{-1} = M^{-1} + W E^{-1} W^T, Eq. mc */
};

enum esd_precond { ESD_PRECOND_NONE = 0, ESD_PRECOND_IC0 = 1 };

enum esd_precision {
  ESD_FP64 = 0,        /* FP64 (the W terms of up to 32 columns in double-float, see esd_solve) */
  ESD_FP32_REFINE = 1  /* FP32 inner PCG inside an FP64 iterative refinement */
};

/* Which iterates a sampled solve (sample_m > 0) keeps, Section 4.2. */
enum esd_sampling {
  ESD_SAMPLING_A = 0,  /* Appendix A: a spread of iterations fixed only at the stop */
  ESD_SAMPLING_B = 1   /* the iterate whose relative residual first reaches tol^(s/(m+1)),
                          s = 1..m (an iteration reaching several levels kept once); FP64 only */
};

typedef struct esd_matrix esd_matrix;
typedef struct esd_solver esd_solver;

/* Message of the last failing call on this thread ("" if none). Library-owned. */
const char* esd_last_error(void);

/* ---------------------------------------------------------------- matrix */

/*
 * ESD_MATRIX_DIAG_SCALE: the library holds the symmetrically Jacobi-scaled matrix
 * A^ = D^-1/2 A D^-1/2, D = diag(A), a^_ij = (a_ij d_i) d_j with d_i = 1/sqrt(a_ii) (the paper
 * scales every test matrix this way, Sections 5.1 and 5.4). Every later call (SpMV, IC(0),
 * solves, W, Ritz values, condition estimates, esd_matrix_set_values) works on A^, so a
 * solve of A x = b is the solve of A^ x^ = d o b followed by x = d o x^ (esd_matrix_diag_scale
 * returns d), with the stopping test on the scaled residual. A diagonal entry that is not
 * positive and finite returns ESD_ERR_INVALID. The finite-volume assembly and its theta
 * gradient refer to the unscaled operator and refuse a scaled matrix (ESD_ERR_STATE);
 * esd_pattern_grad differentiates with respect to the entries of A^.
 */
#define ESD_MATRIX_DIAG_SCALE 1u

/*
 * Create the library's copy of an SPD matrix A (the fixed matrix of the sequence
 * A x_k = b_k, Eq. ak2/ak3) from CSR.
 *   n           rows (= columns), 1 <= n < 2^31 - 64
 *   nnz         entries, rowptr[n]
 *   rowptr      n+1 int32, rowptr[0] = 0, non-decreasing         (device or host)
 *   colind      nnz int32 in [0, n), strictly increasing per row  (device or host)
 *   val         nnz doubles                                       (device or host)
 *   colour_ptr  ncolours+1 int32: rows colour_ptr[c] .. colour_ptr[c+1]-1 form colour c;
 *               colour_ptr[0] = 0, colour_ptr[ncolours] = n (host)
 *   ncolours    1 .. 64; no two rows of one colour may be coupled (multicolour ordering)
 *   flags       0 or ESD_MATRIX_DIAG_SCALE (see there)
 *   stream      cudaStream_t on which all later work is ordered (0 = legacy default stream)
 * Requirements checked on the device: sorted in-range columns, a diagonal entry in every
 * row, a structurally symmetric pattern, no coupling inside a colour. Violations return
 * ESD_ERR_INVALID. Only tril(A) enters the IC(0) factor; SpMV uses A as given.
 * Layout: the rows are re-sliced into a sliced-ELL copy (32-row slices inside each colour).
 */
int esd_create_matrix(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                      const double* val, const int32_t* colour_ptr, int32_t ncolours,
                      uint32_t flags, void* stream, esd_matrix** out);
int esd_matrix_destroy(esd_matrix* A);

/* d_i = 1/sqrt(a_ii) of a matrix created with ESD_MATRIX_DIAG_SCALE, for the diagonal of the
 * values last given (creation or esd_matrix_set_values). d: n doubles, host or device.
 * ESD_ERR_STATE for an unscaled matrix. */
int esd_matrix_diag_scale(const esd_matrix* A, double* d);

/* Dimensions and the colour levels found at creation: a level is a set of colours with
 * no coupling among them, so one launch serves it (forward / backward). */
int esd_matrix_info(const esd_matrix* A, int32_t* n, int64_t* nnz, int32_t* ncolours,
                    int32_t* fwd_levels, int32_t* bwd_levels);

/* Storage the FP32 kernels of the refinement form read (a layout of this library, not in the
 * paper). column_free (host, 3 int32, may be NULL): 1 where A, L, U (in that order) have the
 * column-free copy, built at creation when every 32-row slice has at most 8 distinct
 * (column - lane) values: per slice 8 slot bases (32 bytes) and one 4-byte value per slot
 * and row, 0 where the row lacks that neighbour; 0 where the part keeps its (value, column)
 * pairs of 8 bytes. A's copy has no slot for the diagonal: the FP32 product takes the
 * difference form s_i p_i + sum_j a_ij (p_j - p_i), in which the diagonal multiplies 0.
 * slot_entries (host, 3 int64, may be NULL): the values each copy holds (slots x 32 summed
 * over the slices; 0 without a copy). slices (host, may be NULL): the number of 32-row
 * slices. */
int esd_matrix_layout(const esd_matrix* A, int32_t* column_free, int64_t* slot_entries, int32_t* slices);

/*
 * IC(0) factor M = L L^T on the pattern of tril(A), computed colour by colour in the
 * given order (the paper's incomplete Cholesky preconditioner, Sections 4.4 and 5.3; the
 * fill level is zero). If a pivot is not positive the factor is recomputed for
 * A + s diag(A) with s = 1e-3, 2e-3, 4e-3, ... (at most max_tries attempts in total,
 * the first with s = 0). shift_used (host, may be NULL) receives s.
 * Errors: ESD_ERR_NOT_SPD when every attempt fails.
 */
int esd_factor_ic0(esd_matrix* A, int32_t max_tries, double* shift_used);

/* y = A x (device or host arrays of n doubles). */
int esd_matrix_spmv(esd_matrix* A, const double* x, double* y);

/*
 * New values for A on the pattern given at creation (nnz doubles in that CSR order, host or
 * device). The IC(0) factor is dropped (call esd_factor_ic0 again) and a W built for the
 * old values goes stale (esd_refresh_W); solves refuse to run on either until then.
 */
int esd_matrix_set_values(esd_matrix* A, const double* val);

/*
 * Cell-centred finite-volume diffusion on a structured grid with per-cell coefficient
 * k_c = exp(theta_c): A = inv_dt I + K(theta). An interior face between cells a and b
 * carries T = 2 k_a k_b / (k_a + k_b) / h^2 (harmonic mean) on both diagonals and -T off
 * them; a face on the boundary (Dirichlet) adds 2 k_c / h^2 to the diagonal. Cells are in
 * natural order c = ix + nx (iy + ny iz); cell_row[c] is the matrix row of cell c (the
 * colour-major permutation of the pattern). dims = 2 ignores nz.
 */
typedef struct {
  int32_t dims;
  int32_t nx, ny, nz;
  double h;       /* cell size */
  double inv_dt;  /* 1/dt of backward Euler, 0 for the steady operator */
} esd_fv_grid;

/* Assemble A(theta) on the device into A's values (the pattern must hold the stencil);
 * like esd_matrix_set_values it drops the factor. theta[n], cell_row[n]: host or device.
 * Errors: ESD_ERR_INVALID for a grid that does not match A, a row index outside 0..n-1 or a
 * missing stencil entry (A is then left unchanged). */
int esd_fv_assemble(esd_matrix* A, const esd_fv_grid* g, const double* theta, const int32_t* cell_row);

/*
 * Adjoint gradient of L(x(theta)) for A(theta) x = b: given x and lambda, the solution of the
 * adjoint system A lambda = dL/dx (A is symmetric, so it is one more solve with the same
 * matrix, mode and W), grad_theta[c] = dL/dtheta_c = k_c sum over the faces of c of
 * dL/dT dT/dk_c, with dL/dT = -(lambda_a - lambda_b)(x_a - x_b) on interior faces and
 * -lambda_c x_c 2/h^2 per boundary face. lambda, x: matrix order; theta, grad_theta: natural
 * cell order. dL/db = lambda needs no call. Host or device arrays.
 */
int esd_fv_grad_theta(esd_matrix* A, const esd_fv_grid* g, const double* theta, const int32_t* cell_row,
                      const double* lambda, const double* x, double* grad_theta);

/* z = (L L^T)^{-1} r by colour-ordered forward and backward substitution
 * (requires esd_factor_ic0). */
int esd_matrix_apply_ic(esd_matrix* A, const double* r, double* z);

/*
 * Gradient of a scalar loss with respect to the stored entries of A when x solves
 * A x = b and lambda solves the adjoint system A lambda = dL/dx: dL/da_ij = -lambda_i x_j,
 * written in the order of the CSR given at creation (grad has nnz entries).
 */
int esd_pattern_grad(esd_matrix* A, const double* lambda, const double* x, double* grad);

/* ---------------------------------------------------------------- solver */

typedef struct {
  int32_t precond;     /* esd_precond */
  int32_t maxit_cap;   /* capacity of the alpha/beta history; a solve's maxit <= this */
  int32_t sample_cap;  /* slots reserved for sampled iterates (the paper's m), 0..64 */
  int32_t lmax;        /* sampling method A parameter l_max (m^l_max > N_max); 0 = smallest valid */
  double rank_tol;     /* rank rule for the sampled errors, e.g. 1e-12 */
  int32_t precision;   /* esd_precision */
  double inner_tol;    /* ESD_FP32_REFINE: residual reduction of each FP32 inner solve */
  int32_t max_outer;   /* ESD_FP32_REFINE: refinement steps allowed */
  int32_t resume_direction; /* ESD_FP32_REFINE: 1 = every step resumes CG with the kept search
                               direction (residual replacement), 0 = every step restarts CG */
  int32_t sampling;    /* esd_sampling: which iterates a sampled solve keeps */
} esd_params;

/* Default parameters: IC(0), maxit_cap 20000, sample_cap 32, lmax 0, rank_tol 1e-12, FP64,
 * sampling method A;
 * for ESD_FP32_REFINE inner_tol 0.1, max_outer 60, resume_direction 1. */
void esd_params_default(esd_params* p);

int esd_solver_create(esd_matrix* A, const esd_params* params, esd_solver** out);
int esd_solver_destroy(esd_solver* S);

/* Select the iteration: ESD_PLAIN, ESD_DEFLATION or ESD_SUBSPACE_CORRECTION. The last two
 * need W (esd_sample_and_build_W or esd_set_W), otherwise ESD_ERR_STATE. */
int esd_set_mode(esd_solver* S, int32_t mode);

/*
 * Solve A x = b to ||b - A x||_2 <= tol ||b||_2 (the paper's criterion, Section 5.1).
 *   b         n doubles (device or host), unchanged
 *   x         n doubles (device or host): initial guess on entry, solution on exit
 *   tol       relative tolerance > 0
 *   maxit     1 .. maxit_cap
 *   sample_m  0, or 1 .. sample_cap: store iterates by the solver's sampling method (A,
 *             Appendix A, needs m >= 2; or B, Section 4.2) for a following
 *             esd_sample_and_build_W. Not allowed in deflation mode (its iterates live in
 *             the deflated space): ESD_ERR_STATE.
 *   iters     (host, may be NULL) alpha steps taken
 *   relres    (host, may be NULL) final ||r_i||/||b|| of the recursive residual; in
 *             deflation mode r_i = P^T (b - A x_i), which equals the true residual of the
 *             returned x (Eq. x1/x2)
 * Plain / SC mode: PCG as in Algorithm "PCG with condition number estimation", with its
 * power method once esd_power_start has been called (see there). Deflation: Algorithm
 * "Deflated PCG" with beta = +rho_{i+1}/rho_i and the final x = P x_i + W E^{-1} W^T b.
 * b = 0 gives x = 0 and 0 iterations.
 * Arithmetic of the FP64 form: FP64 throughout, except that with up to 32 (padded) columns of
 * W the deflation and subspace-correction terms ((AW)^T p, AW y, W^T r, W u) are formed in
 * double-float arithmetic on the FP32 pipe (float pairs, about 48 significant bits; terms
 * 2^-100 below the largest dropped), below FP64's own rounding of these n-term sums.
 * The whole solve is one CUDA graph launch (a device-side while loop); the call
 * synchronises once at the end to return iters and relres.
 * Precision ESD_FP32_REFINE (not in the paper): x is refined in FP64. Each step forms
 * r = b - A x in FP64; when ||r|| > tol ||b|| it solves A d = r with the selected mode in
 * FP32 (FP32 matrix, factor, W and AW, FP32-accumulated dot products; E^{-1} stays FP64)
 * to ||r_inner|| <= max(inner_tol ||r||, tol ||b|| / 2), then x += d in FP64; at most
 * max_outer steps. With resume_direction the inner CG state carries over from step to step
 * (only the residual is replaced by the FP64 one), so the steps form one CG run; otherwise
 * each inner solve starts afresh. Both loops run on the device (nested while nodes). iters
 * counts the inner iterations (and maxit bounds them: per inner solve when restarting, in
 * total when resuming); relres is the FP64 true residual. Sampling (sample_m > 0) stores
 * FP64 iterates (the FP64 x plus the inner iterate) of the first inner solve, or of the whole
 * run when resuming.
 * Errors: ESD_ERR_MAXIT (x = last iterate), ESD_ERR_BREAKDOWN, ESD_ERR_STATE.
 */
int esd_solve(esd_solver* S, const double* b, double* x, double tol, int32_t maxit,
              int32_t sample_m, int32_t* iters, double* relres);

/*
 * Two systems A x_1 = b_1 and A x_2 = b_2 with the same matrix, solved together (not in the
 * paper: a way of running two solves of a sequence that need only the same earlier solution,
 * such as the adjoint of system t and the forward solve of system t + 1, which both need
 * x_t). Each system runs its own refinement-form solve exactly as esd_solve does it (plain
 * PCG with IC(0), FP32 inner runs, FP64 refinement, same tol and maxit, no sampling), with its
 * own solver's state. In every refinement step the inner iterations of both share each pass
 * over the matrix and its factor while both inner runs go on; the one left then goes on with
 * the single kernels. The two trajectories equal their single runs up to the rounding of the
 * FP32 dot products, whose per-thread partial sums cover other rows.
 * S1, S2: two distinct solvers on the same matrix (and preconditioning matrix), both in
 * ESD_FP32_REFINE and ESD_PLAIN with IC(0), no power method. b_k, x_k: n doubles each, host
 * or device, x_k the start vector on input and the solution on output. iters_k, relres_k
 * (host, may be NULL): as esd_solve's, per system; each solver's esd_last_solve_info and
 * esd_true_relres describe its system afterwards. paired (host, may be NULL): iterations
 * run by the paired kernels (each advanced both systems), over all refinement steps. The first call for a pair builds its graph
 * (kept in S1 while neither solver's graphs are rebuilt).
 * Errors: ESD_ERR_STATE when the pair cannot run these kernels (the message says why: the
 * staged kernels are off, rows wider than 8 entries, more than 16 forward colour levels, ...);
 * otherwise as esd_solve, the first failing system's code (the message names it).
 */
int esd_solve_pair(esd_solver* S1, esd_solver* S2, const double* b1, double* x1, const double* b2, double* x2,
                   double tol, int32_t maxit, int32_t* iters1, double* relres1, int32_t* iters2, double* relres2,
                   int32_t* paired);

/*
 * Measurement of the pair solve's kernels: reps paired iterations of the FP32 inner PCG on
 * A d = b_1 and A d = b_2 from d = x_1, x_2 (rounded to FP32), launched one by one with CUDA
 * events between them, as esd_profile_iterations does for one system (tolerance 0). S1, S2
 * as esd_solve_pair asks (same errors); ms, names, cap, count as esd_profile_iterations;
 * x_1, x_2 (device or host) receive the FP64 iterates after reps steps.
 */
int esd_profile_pair_iterations(esd_solver* S1, esd_solver* S2, const double* b1, double* x1, const double* b2,
                                double* x2, int32_t reps, double* ms, char* names, int32_t cap, int32_t* count);

/* ||b - A x|| / ||b|| of the last solve, recomputed in FP64 from the returned x. */
int esd_true_relres(esd_solver* S, double* relres);

/*
 * The last solve in numbers (host pointers, any may be NULL): iters = CG iterations (in the
 * refinement form the inner FP32 iterations of all steps), outer_steps = refinement steps
 * (0 in FP64 form), first_inner = iterations of the first inner solve, the one sampling
 * reads (= iters in FP64 form), restarts = resumed steps that restarted the search
 * direction because the inner residual had drifted from the true one by more than half of it,
 * max_gap = the largest such relative drift seen, true_relres = ||b - A x||/||b|| in FP64,
 * status = the solve's return code.
 */
int esd_last_solve_info(esd_solver* S, int32_t* iters, int32_t* outer_steps, int32_t* first_inner,
                        int32_t* restarts, double* max_gap, double* true_relres, int32_t* status);

/*
 * Build W from the iterates stored by the last sampling solve (Section 4.2):
 * e_s = x - x~_s (Eq. ek) for every filled slot, columns normalised, the rank
 * mbar = #{eig(G) > rank_tol max eig(G)} of G = Ehat^T Ehat, an orthonormal basis Q of
 * their span (Eq. ekd; CholeskyQR2 when full rank, else SVQB then one CholeskyQR pass),
 * then with theta = +inf W = Q, or with finite theta the Ritz vectors Q t_i of
 * Q^T A Q t = lambda t with lambda < theta (Eq. Rayleigh-Ritz, bk). Also AW = A W,
 * E = W^T A W and E^{-1}, all in FP64 on the device.
 *   m_kept  (host, may be NULL) number of columns of W
 * Errors: ESD_ERR_STATE (no sampled solve), ESD_ERR_RANK, ESD_ERR_CHOL_E.
 */
int esd_sample_and_build_W(esd_solver* S, double theta, int32_t* m_kept);

/* Use a caller-supplied W (n x m column-major doubles, device or host, 1 <= m <= 64,
 * columns linearly independent); AW, E and E^{-1} are built as above. */
int esd_set_W(esd_solver* S, const double* W, int32_t m);

/*
 * Precondition with the IC(0) factor of P instead of A's own: M = L_P L_P^T. P holds the same
 * rows in the same colour-major order as A (same n and colour_ptr, so the same 32-row
 * slices) and is factored (esd_factor_ic0). Its own couplings set the colour levels of the
 * substitutions. The paper's parallel solver uses block-Jacobi IC (Section 5.3): P is the
 * block-diagonal part of A, and colours that are coupled only across blocks share a launch.
 * The products with A (SpMV, residuals, W) still use A. P must stay alive and factored
 * while the solver uses it; NULL returns to A's factor.
 * Errors: ESD_ERR_INVALID for other rows or colours, ESD_ERR_STATE for an unfactored P.
 */
int esd_solver_set_precond_matrix(esd_solver* S, esd_matrix* P);

/*
 * Switch an existing solver between ESD_FP64 and ESD_FP32_REFINE (the precision of
 * esd_params) and set the inner tolerance of the refinement form (0 < inner_tol < 1; ignored
 * for ESD_FP64). The first switch to the refinement form allocates its buffers and the FP32
 * copies of the matrix. A W already built is kept: switching to the refinement form rounds it
 * to FP32 and forms AW, E and E^-1 again for that W (as esd_set_W would); switching back keeps
 * that W. Errors: ESD_ERR_INVALID for sampling method B with the refinement form,
 * ESD_ERR_STATE while the power method runs (it needs FP64 solves).
 */
int esd_set_precision(esd_solver* S, int32_t precision, double inner_tol);

/* AW, E = W^T A W, E^-1 and the Ritz values formed again for the current W and the current
 * values of A (after esd_matrix_set_values / esd_fv_assemble). ESD_ERR_STATE without W. */
int esd_refresh_W(esd_solver* S);

/* Copy W, AW (n x m column-major) and E (m x m row-major) out; any pointer may be NULL. */
int esd_get_W(esd_solver* S, double* W, double* AW, double* E, int32_t* m);

/* Ritz values of the current W (eigenvalues of E when W is orthonormal), ascending. */
int esd_ritz_values(esd_solver* S, double* out, int32_t cap, int32_t* count);

/*
 * Condition number estimate from the last solve: the extreme eigenvalues of the Lanczos
 * tridiagonal matrix assembled from its CG coefficients, T_jj = 1/alpha_j +
 * beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j. They estimate the spectrum
 * of the (preconditioned, deflated) operator of that solve; kappa = lmax/lmin.
 * ritz_min (may be NULL) receives the smallest Ritz value of W (the paper's lambda_min
 * estimate, Section 5.4) or NaN when there is no W.
 */
int esd_estimate_cond(esd_solver* S, double* lmin, double* lmax, double* kappa, double* ritz_min);

/*
 * Power method of Algorithm "PCG with condition number estimation" (Section 5.4): from a start
 * vector v_0, every CG iteration of the following FP64 plain or subspace-correction solves
 * also forms v_i = A v_{i-1} / ||A v_{i-1}||_2 in the same pass over the matrix as q = A p
 * (one read of each entry serves both products). The vector carries over from solve to
 * solve (and through esd_profile_iterations) until the next esd_power_start. A solve in
 * deflation mode is refused (ESD_ERR_STATE) while it runs; its iterations would not advance it.
 *   v0   n doubles (device or host), any nonzero finite vector (the paper: a unit random
 *        vector); it is normalised here. NULL stops the power method.
 * Errors: ESD_ERR_STATE for an ESD_FP32_REFINE solver, ESD_ERR_INVALID for a zero or
 * non-finite v0 (the method is then off).
 * Costs per iteration: nnz FMAs and 16 bytes per row (read v_{i-1}, write v_i) on top of
 * the SpMV.
 */
int esd_power_start(esd_solver* S, const double* v0);

/*
 * The power method's estimate lambda_max = (v_k, A v_k) of the current unit vector v_k, the
 * paper's largest-eigenvalue estimate; with the smallest Ritz value of the errors sampled in
 * the same solve (esd_sample_and_build_W with theta = +inf, then esd_ritz_values) it gives the
 * paper's kappa = lambda_max / lambda_min. One pass over A; no iteration is taken.
 *   lmax   (host, may be NULL) the estimate
 *   steps  (host, may be NULL) k, the products taken since esd_power_start
 *   v      (may be NULL) n doubles (device or host) receiving v_k
 * Errors: ESD_ERR_STATE when not started, ESD_ERR_BREAKDOWN when the vector vanished or
 * overflowed (A v = 0 for a singular A, or a non-finite product).
 */
int esd_power_estimate(esd_solver* S, double* lmax, int32_t* steps, double* v);

/*
 * The paper's condition number estimate (Algorithm "PCG with condition number estimation",
 * Section 5.4): kappa = lambda_max / lambda_min with lambda_max = (v_k, A v_k) of the power
 * method (as esd_power_estimate) and lambda_min the smallest Ritz value of the current W
 * (esd_sample_and_build_W with theta = +inf on the sampled solve, Eq. Rayleigh-Ritz).
 *   lmax, lmin, kappa  (host, any may be NULL)
 * Errors: ESD_ERR_STATE without W or without the power method, ESD_ERR_BREAKDOWN as
 * esd_power_estimate, ESD_ERR_CHOL_E when the smallest Ritz value is not positive.
 */
int esd_paper_cond_estimate(esd_solver* S, double* lmax, double* lmin, double* kappa);

/* alpha_j and beta_j of the last solve (host arrays of cap entries). */
int esd_get_history(esd_solver* S, double* alpha, double* beta, int32_t cap, int32_t* count);

/* Sampled slots of the last sampling solve: iteration held by each slot (0 = empty). */
int esd_get_samples(esd_solver* S, double* samples, int32_t* slot_iter, int32_t cap, int32_t* m);

/*
 * Measurement: run reps iterations of the current mode on A x = b starting from x, the same
 * kernels the solve graph holds but launched one by one with CUDA events between them, and
 * return each kernel's average device time in launch order (the tolerance is taken as 0, so
 * the iterations do not stop early).
 *   ms     host array of cap doubles: average milliseconds per kernel launch
 *   names  host buffer of 32*cap chars (may be NULL): NUL-terminated kernel names, 32 bytes each
 *   count  (host) kernels in one iteration
 * x (device or host) receives the iterate after reps steps.
 */
int esd_profile_iterations(esd_solver* S, const double* b, double* x, int32_t reps, double* ms,
                           char* names, int32_t cap, int32_t* count);

/*
 * Condition estimate that allocates no device memory. The paper has no counterpart: it exists
 * for callers that cannot call cudaMalloc, for example code whose whole device memory has
 * been handed to another allocator, or a time-stepping loop that must not block on the
 * implicit device synchronisation an allocation can cause. It returns what esd_estimate_cond
 * returns (without the Ritz value), from CG coefficients the caller supplies.
 *   alpha  device array of k doubles, beta device array of k-1 doubles (as esd_get_history
 *          returns them; beta may be NULL when k = 1)
 *   k      1 .. ESD_NOALLOC_MAX_K; a larger k returns ESD_ERR_INVALID before any launch
 *   out    device array of 3 doubles: lambda_min, lambda_max, kappa
 *   stream cudaStream_t of the launch (0 = legacy default stream); the call does not wait
 * alpha, beta and out must be device (or managed) memory of the current device, holding at
 * least k, k-1 and 3 doubles; a pointer that is not (a host array, another GPU's memory)
 * returns ESD_ERR_INVALID before any launch. The lengths cannot be checked here: the Python
 * binding checks them.
 * Scratch: a file-scope device array of 2 * ESD_NOALLOC_MAX_K doubles (512 KB), which every
 * GPU that loads the library holds until the process exits. The first call on a device, with
 * that device current, looks up the array's device address; make that first call before any
 * stream capture. All calls share the array, so calls that overlap on the GPU (unordered
 * streams) race; order them on one stream. Nothing needs clearing: each call writes the k
 * entries it reads.
 */
#define ESD_NOALLOC_MAX_K 32768
int esd_lanczos_extremes_noalloc(const double* alpha, const double* beta, int32_t k, double* out,
                                 void* stream);

/* b = x_prev * inv_dt + s, the backward-Euler right-hand side of the next system. */
int esd_backward_euler_rhs(esd_solver* S, const double* x_prev, const double* s, double inv_dt,
                           double* b);

#ifdef __cplusplus
}
#endif

#endif /* ESDCG_H */
