/*
 * iga_fd.h -- C ABI of the GB300 (sm_103a) library for IGA collocation of the
 * Poisson problem solved by GMRES preconditioned with fast diagonalization (FD).
 *
 * Method: M. Tani, "A preconditioning strategy for linear systems arising from
 * nonsymmetric schemes in isogeometric analysis", arXiv:1705.04384.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Degrees of freedom: n = n_elem + p - 2 per direction (Sec. 2.1, eq. space:
 *   interior basis B_1..B_n of the open knot vector with n_elem uniform elements,
 *   simple interior knots, C^{p-1}); N = n^d.
 * - Vector layout: one value per DOF / collocation point in the scalar order of
 *   eq. (space), i = i_1 + n i_2 + n^2 i_3 (0-based), i_1 fastest, contiguous,
 *   IEEE binary64.
 * - "_dev" pointers are CUDA device pointers on the device that was current at
 *   iga_setup; "_host" pointers are ordinary host memory.  The CALLER owns every
 *   pointer it passes; the library never frees or retains them after returning.
 * - The LIBRARY owns all state behind an iga_handle (1D factors, eigen-factors,
 *   geometry coefficients, Krylov workspace, CUDA graphs); iga_destroy frees it.
 *   1D factors are cached per (n_elem, p) and shared between handles.
 * - All device work is ordered on the stream given to iga_setup (NULL = legacy
 *   default stream).  Calls returning results to host memory synchronize that
 *   stream before returning; iga_apply_operator and iga_precond_apply are
 *   asynchronous (stream-ordered) and return right after enqueueing.
 * - A handle must not be used from two host threads at once.
 * - Errors: every call returns an iga_status; nothing is thrown across the ABI
 *   and nothing calls exit().  iga_last_error() gives a message for the most
 *   recent failure on the calling thread.  On IGA_ERR_CUDA the handle should be
 *   destroyed.
 */
#ifndef IGA_FD_H
#define IGA_FD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iga_ctx *iga_handle;

typedef enum {
  IGA_OK = 0,
  IGA_ERR_INVALID_ARG = 1,        /* bad size, pointer or enum value                  */
  IGA_ERR_OOM = 2,                /* device or host allocation failed                 */
  IGA_ERR_CUDA = 3,               /* a CUDA runtime / cuSOLVER call failed            */
  IGA_ERR_NOT_DIAGONALIZABLE = 4, /* Remark 1 violated: complex eigenvalues or
                                     ill-conditioned eigenvector matrix               */
  IGA_ERR_NO_CONVERGENCE = 5,     /* tolerance not reached within max_iter            */
  IGA_ERR_DEVICE_TIMEOUT = 6,     /* a bounded device-side wait gave up               */
  IGA_ERR_NAN = 7,                /* non-finite value in the right-hand side or solve */
  IGA_ERR_UNSUPPORTED = 8         /* valid request this build does not implement      */
} iga_status;

/* Geometry map F : [0,1]^d -> Omega (Sec. 2.1, single patch).  Analytic maps:
 *  IDENTITY          Omega = [0,1]^d; then A_C = P_C (eqs. colloc2D / colloc3D).
 *  QUARTER_ANNULUS   d = 2: x = r cos(pi eta/2), y = r sin(pi eta/2),
 *                    r = r_inner + (r_outer - r_inner) xi  (Sec. 5 quarter of ring);
 *                    d = 3: the same ring extruded, z = zeta.
 *  REVOLVED_ANNULUS  d = 3: the ring turned by pi/2 * zeta about the axis through
 *                    (-1,-1,-1) with direction (0,1,0) (Sec. 5 revolved ring).       */
typedef enum {
  IGA_GEOM_IDENTITY = 0,
  IGA_GEOM_QUARTER_ANNULUS = 1,
  IGA_GEOM_REVOLVED_ANNULUS = 2
} iga_geom_kind;

typedef struct {
  int kind;       /* iga_geom_kind */
  double r_inner; /* ring radii (ignored for IDENTITY); 0 < r_inner < r_outer */
  double r_outer;
  /* Constant wind w (physical components; entries past d ignored).  Zero: the Poisson
   * problem of eq. (poisson).  Nonzero: the convection-diffusion operator
   * -Lap + w . grad of Sec. 3.2 (eq. convection), collocated like -Lap, and the FD
   * preconditioner of eq. (convec_prec_2) in collocation form, direction l factor
   * K_l + H_l = -B''_l + w_l B'_l.  Requires precision FP64 or NONE.  The FD needs the
   * shifted pencils to be diagonalizable with a well-conditioned eigenvector basis:
   * on these meshes that holds for |w_l| up to about 10 (NOT_DIAGONALIZABLE beyond). */
  double wind[3];
} iga_geometry;

/* Precision of the preconditioner apply (Sec. 4 FD).  FP64: plain GMRES with an
 * FP64 FD.  TF32 / BF16: FD mode products on the tcgen05 tensor cores with FP32
 * accumulation inside flexible GMRES; operator, orthogonalization, least squares
 * and eigen-factors stay FP64.  TF32X3: the same with error-compensated TF32 -- every
 * operand is split into a TF32 part and the TF32 rounding of its remainder, and each
 * product sums hi*hi + hi*lo + lo*hi in FP32 (three MMAs per step), which brings the FD
 * close to FP32 accuracy (and the flexible GMRES close to the FP64 form's step count) for
 * about the cost of the latency-bound TF32 products.  FP64_TC: the FP64 form (plain GMRES,
 * FP64 FD to FP64 accuracy) with the FD mode products on the BF16 tensor cores by exact
 * integer slice products (error-free splitting of Ozaki et al. 2012: 8 digits of 7 bits
 * per value, exact FP32 sums, recombined exactly before one rounding); n <= 148, no wind.
 * NONE: no preconditioner (P = I).                                                     */
typedef enum {
  IGA_PREC_FP64 = 0,
  IGA_PREC_TF32 = 1,
  IGA_PREC_BF16 = 2,
  IGA_PREC_NONE = 3,
  IGA_PREC_TF32X3 = 4,
  IGA_PREC_FP64_TC = 5
} iga_precision;

/* Discretization scheme of iga_setup_scheme.
 *  COLLOCATION   isogeometric collocation at the Greville points (Sec. 2.2, eq.
 *                collocationsystem); preconditioner P_C of eq. colloc2D / colloc3D.
 *  WQ_GALERKIN   Galerkin with weighted quadrature (Sec. 2.3, eq. WQapprox): test
 *                function i's univariate rules w^{(s,t)} are exact on the spline space
 *                (every overlapping basis function, value or derivative), live on the
 *                quadrature points in its support and have minimum 2-norm; quadrature
 *                points are the element end points and midpoints, with p equispaced
 *                interior points in the first and last element; coefficients Q =
 *                det(J) J^{-1} J^{-T} (eq. Q, K = I).  Preconditioner P_wq = P_G of eq.
 *                wq2D / wq3D (univariate Galerkin M, K: the symmetric FD of Sec. 4).  No
 *                wind.  The right-hand side is the caller's (see iga_wq_load).          */
typedef enum { IGA_SCHEME_COLLOCATION = 0, IGA_SCHEME_WQ_GALERKIN = 1 } iga_scheme;

/* Factor selectors for iga_get_factor (all n x n row-major unless noted).  For a
 * WQ_GALERKIN problem M and K are the univariate Galerkin matrices of eq. (univariateWQ). */
typedef enum {
  IGA_FACTOR_TAU = 0,    /* Greville points tau_i, eq. (greville): n values        */
  IGA_FACTOR_M = 1,      /* (M)_ij = B_j(tau_i), eq. (univariatecolloc)            */
  IGA_FACTOR_B1 = 2,     /* B'_j(tau_i)                                            */
  IGA_FACTOR_K = 3,      /* (K)_ij = -B''_j(tau_i), eq. (univariatecolloc)         */
  IGA_FACTOR_LAMBDA = 4, /* eigenvalues D of M^{-1}K, eq. (eigendecomposition), asc */
  IGA_FACTOR_U = 5,      /* eigenvectors U (unit 2-norm columns)                   */
  IGA_FACTOR_VT = 6      /* V^T = (M U)^{-1}  (Sec. 4, V := (M U)^{-T})             */
} iga_factor;

/* Build a problem: 1D spaces and collocation factors (Sec. 2.1-2.2), geometry
 * coefficients of the pulled-back operator at the collocation points F(tau_I),
 * and the FD eigen-factors of eq. (eigendecomposition) for each direction.
 *   d          2 or 3
 *   n_elem     elements per direction, >= 3 (so that n >= p + 1)
 *   p          spline degree, 2..6
 *   geom       geometry (not retained)
 *   precision  iga_precision
 *   stream     cudaStream_t to order all work on (NULL = default stream)
 *   out        receives the handle
 * Synchronous.  Errors: INVALID_ARG, OOM, CUDA, NOT_DIAGONALIZABLE.           */
iga_status iga_setup(int d, int n_elem, int p, const iga_geometry *geom,
                     int precision, void *stream, iga_handle *out);

/* iga_setup with a choice of discretization (iga_scheme); iga_setup is scheme
 * COLLOCATION.  Same arguments, ownership and errors as iga_setup; WQ_GALERKIN rejects a
 * nonzero wind (INVALID_ARG).                                                */
iga_status iga_setup_scheme(int d, int n_elem, int p, const iga_geometry *geom, int scheme,
                            int precision, void *stream, iga_handle *out);

/* n (DOFs per direction) and N = n^d.  Either pointer may be NULL. */
iga_status iga_dims(iga_handle h, int *n, long long *N);

/* Physical collocation points F(tau_I) (eq. collocation), written as N x d
 * row-major doubles (point I at xyz_host[I*d .. I*d+d-1]) in DOF order.  The
 * right-hand side of eq. (collocationsystem) is f evaluated at these points.
 * UNSUPPORTED for a WQ_GALERKIN problem.                                      */
iga_status iga_collocation_points(iga_handle h, double *xyz_host);

/* WQ_GALERKIN problems only (UNSUPPORTED otherwise): nq quadrature points per direction and
 * Nq = nq^d; the physical quadrature points F(x_q), Nq x d row-major, direction 1 fastest
 * (the order of the values iga_wq_load takes).                               */
iga_status iga_quadrature_dims(iga_handle h, int *nq, long long *Nq);
iga_status iga_quadrature_points(iga_handle h, double *xyz_host);

/* WQ_GALERKIN problems only: the load vector f_I = sum_q w^{00}_{Iq} |det J(x_q)| g_q, the
 * weighted-quadrature approximation of int g(F(xi)) B_I(xi) |det J(xi)| dxi (Sec. 2.3: the
 * right-hand side of eq. WQsystem "by using again the WQ approach").  g_dev: Nq doubles
 * (values of the source at iga_quadrature_points); f_dev: N doubles.  Stream-ordered,
 * asynchronous.  Errors: INVALID_ARG, UNSUPPORTED (collocation problem), CUDA. */
iga_status iga_wq_load(iga_handle h, const double *g_dev, double *f_dev);

/* Copy a 1D factor of direction dir (0..d-1) to host memory (see iga_factor for
 * shapes).  Synchronous.                                                     */
iga_status iga_get_factor(iga_handle h, int dir, int which, double *out_host);

/* Au = A_C u: the collocation matrix of eq. (collocationsystem), applied matrix-
 * free by sum factorization of the banded 1D factors and a pointwise contraction
 * with the geometry coefficients.  For a WQ_GALERKIN problem Au = A_wq u (eq.
 * WQapprox), by sum factorization onto the quadrature grid and back (banded basis
 * values / derivatives at the points, the Q field, banded univariate rules).
 * u_dev, Au_dev: N doubles, must not overlap.  Stream-ordered, asynchronous.  */
iga_status iga_apply_operator(iga_handle h, const double *u_dev, double *Au_dev);

/* s = P^{-1} b by the FD method, eq. (FD2D) (d = 2) or eq. (FD3D) (d = 3), in the
 * handle's precision (TF32/BF16 round the input and intermediates; the result is
 * returned in binary64).  For IGA_PREC_NONE it copies b.  b_dev, s_dev: N doubles,
 * must not overlap.  Stream-ordered, asynchronous.                           */
iga_status iga_precond_apply(iga_handle h, const double *b_dev, double *s_dev);

/* Solve A_C x = rhs (eq. collocationsystem) by unrestarted GMRES (Sec. 3, Saad &
 * Schultz), right-preconditioned with P^{-1} (flexible GMRES for TF32/BF16),
 * until |g_{k+1}| <= tol * ||rhs||_2 or max_iter iterations.
 *   rhs_dev       N doubles (device)
 *   x_dev         N doubles (device): the solution on return; if use_x0 != 0 it
 *                 holds the initial guess on entry, else x0 = 0
 *   tol           relative residual target (> 0 or 0 to run max_iter steps)
 *   max_iter      1..4096
 *   iters         (host, may be NULL) iterations performed
 *   res_hist_host (host, may be NULL) max_iter + 1 doubles: estimated relative
 *                 residuals |g_j| / ||rhs||, j = 0..iters
 *   true_relres   (host, may be NULL) ||rhs - A_C x|| / ||rhs|| evaluated in FP64
 * Returns IGA_OK, IGA_ERR_NO_CONVERGENCE (x and outputs still valid), IGA_ERR_NAN
 * (non-finite rhs or breakdown), or an error.  Synchronizes the stream.      */
iga_status iga_solve(iga_handle h, const double *rhs_dev, double *x_dev, int use_x0,
                     double tol, int max_iter, int *iters, double *res_hist_host,
                     double *true_relres);

/* iga_solve for nrhs right-hand sides of the same problem at once.  Each right-hand
 * side has its own Krylov space, rotations and stopping test (the same GMRES as
 * iga_solve, bitwise identical per right-hand side); they advance in lockstep so
 * that every operator pass and FD mode product serves all of them in one launch.
 *   nrhs          1..1024
 *   rhs_dev       nrhs x N doubles, right-hand side r at rhs_dev + r*N
 *   x_dev         nrhs x N doubles (solutions; initial guesses if use_x0)
 *   iters         (host, may be NULL) nrhs iteration counts
 *   res_hist_host (host, may be NULL) nrhs x (max_iter + 1) residual estimates
 *   true_relres   (host, may be NULL) nrhs FP64 true relative residuals
 *   status        (host, may be NULL) nrhs per-right-hand-side iga_status values
 * Returns IGA_ERR_NAN if any right-hand side hit a non-finite value, else
 * IGA_ERR_NO_CONVERGENCE if any missed tol, else IGA_OK.  Synchronizes the stream. */
iga_status iga_solve_multi(iga_handle h, int nrhs, const double *rhs_dev, double *x_dev,
                           int use_x0, double tol, int max_iter, int *iters,
                           double *res_hist_host, double *true_relres, int *status);

/* Asynchronous form of iga_solve_multi: enqueues the whole solve (one CUDA graph
 * launch plus copies) on the handle's stream and returns.  At most one solve per
 * handle may be in flight; rhs_dev and x_dev must stay valid until it completes.
 * iga_solve_ready sets *ready to 1 once the solve has finished (never blocks);
 * iga_solve_collect waits for it and returns its results and status exactly as
 * iga_solve_multi does.  Handles on different streams run concurrently.       */
iga_status iga_solve_async(iga_handle h, int nrhs, const double *rhs_dev, double *x_dev,
                           int use_x0, double tol, int max_iter);
iga_status iga_solve_ready(iga_handle h, int *ready);
iga_status iga_solve_collect(iga_handle h, int *iters, double *res_hist_host, double *true_relres,
                             int *status);

/* Batched form: nprob independent problems (distinct handles, ideally each on its
 * own stream) with nrhs[q] right-hand sides each, x0 = 0.  All solves are enqueued
 * first (one graph launch per problem, all right-hand sides of a problem in
 * lockstep) and then collected, so the problems overlap on the device.
 *   rhs_dev[q], x_dev[q]     nrhs[q] x N_q doubles (device)
 *   iters, true_relres, status  (host, may be NULL) sum(nrhs) entries, problem-major
 *   res_hist_host            (host, may be NULL) sum(nrhs) x (max_iter + 1) residual
 *                            estimates |g_j| / ||rhs||, problem-major, right-hand side r
 *                            of the whole batch at res_hist_host + r (max_iter + 1);
 *                            entries past that right-hand side's iterations are 0
 * Returns the worst status as iga_solve_multi does.                          */
iga_status iga_solve_batched(int nprob, const iga_handle *handles, const int *nrhs,
                             const double *const *rhs_dev, double *const *x_dev, double tol,
                             int max_iter, int *iters, double *res_hist_host,
                             double *true_relres, int *status);

/* iga_solve with host buffers: copies rhs_host (N doubles) to the device, solves
 * with x0 = 0, and copies the solution to x_host (N doubles).  Same outputs and
 * errors as iga_solve.  Synchronous.                                         */
iga_status iga_solve_host(iga_handle h, const double *rhs_host, double *x_host,
                          double tol, int max_iter, int *iters, double *res_hist_host,
                          double *true_relres);

/* Kernel launches of one iga_solve with this handle: fixed + per_iteration * iters.
 * Counts this library's kernels in the captured solve graph (prologue + epilogue,
 * and one Arnoldi step); builds the graph if no solve has run yet.           */
iga_status iga_launch_counts(iga_handle h, int *fixed, int *per_iteration);

/* Which kernel runs the mode products of this handle's FD solve for nrhs right-hand sides
 * (eq. FD2D / FD3D): *kind = IGA_FD_KERNEL_FOLD_MMA (folded products, FP64 mma.sync),
 * IGA_FD_KERNEL_FOLD_FMA (folded products, FP64 FMAs), IGA_FD_KERNEL_DENSE_MMA (pencils
 * without reflection parity, FP64 mma.sync), IGA_FD_KERNEL_TENSOR_CORE (tcgen05, the
 * TF32 / BF16 / TF32X3 precision forms) or IGA_FD_KERNEL_FP64_SLICES (tcgen05 BF16 slice
 * products, the FP64_TC form).  The FP64 choice depends on the size (more rows favour the
 * FMA kernel); IGA_FD64=fma|mma in the environment forces one.  Errors:
 * IGA_ERR_INVALID_ARG for a null handle or kind, nrhs < 1, or an unpreconditioned handle. */
typedef enum {
  IGA_FD_KERNEL_FOLD_MMA = 0,
  IGA_FD_KERNEL_FOLD_FMA = 1,
  IGA_FD_KERNEL_DENSE_MMA = 2,
  IGA_FD_KERNEL_TENSOR_CORE = 3,
  IGA_FD_KERNEL_FP64_SLICES = 4
} iga_fd_kernel_kind;
iga_status iga_fd_kernel(iga_handle h, int nrhs, int *kind);

/* Algorithmic FLOPs of one iga_apply_operator on one vector, counted from the handle's
 * pass plan: 2 per stored band entry of every banded mode product (sum factorization of
 * eq. collocation, or of eq. WQapprox: expansion onto the quadrature grid and contraction
 * by the WQ rules), plus 2 per contracted collocation term and 1 per quadrature point of a
 * Q-weighted WQ term.  Errors: IGA_ERR_INVALID_ARG for a null handle or flops.            */
iga_status iga_operator_flops(iga_handle h, double *flops);

/* s = P^{-1} b by the FP64 FD method, eq. (FD2D) / (FD3D), for callers that cannot
 * allocate device memory when they apply the preconditioner (a fixed memory budget
 * reserved up front, an allocator-free real-time loop, or a host whose own allocator owns
 * the device).  The paper has no counterpart; this is a deployment variant.  No handle is
 * needed and nothing is allocated: the two intermediate tensors live in a static device
 * array of 2 x 2^21 doubles (32 MiB) inside the library.  That array is reserved on a
 * device when the library's module is loaded there: with CUDA's default lazy loading at
 * the first call of this function on that device, with CUDA_MODULE_LOADING=EAGER on every
 * device the library initialises; it stays reserved until the process exits.
 *   d          2 or 3;  n  DOFs per direction; N = n^d must be <= 2097152
 *   Vt_dev     d matrices V_l^T = (M_l U_l)^{-1}, n x n row-major each, direction l at
 *              Vt_dev + l n^2 (iga_get_factor IGA_FACTOR_VT of direction l)
 *   U_dev      d matrices U_l, n x n row-major, direction l at U_dev + l n^2
 *              (IGA_FACTOR_U of direction l)
 *   lam_dev    d x n eigenvalues, direction l at lam_dev + l n (IGA_FACTOR_LAMBDA)
 *              Each direction has its own factors: the Poisson pencils of all directions
 *              coincide on these uniform meshes, the wind-shifted pencils of Sec. 3.2 do not.
 *   b_dev, s_dev  N doubles, must not overlap; all pointers are the caller's
 *   stream     cudaStream_t (NULL = default stream); asynchronous, stream-ordered
 * The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.  All
 * calls share the one array: calls that overlap on the GPU (other streams, other host
 * threads) race on it and give wrong results.  The array needs no clearing: every
 * entry is written before it is read.
 * Errors: INVALID_ARG (bad d, n, null pointer, N above the limit), CUDA.      */
iga_status iga_precond_apply_noalloc(int d, int n, const double *Vt_dev, const double *U_dev,
                                     const double *lam_dev, const double *b_dev, double *s_dev,
                                     void *stream);

/* Solve A_C x = b with BiCGStab (van der Vorst 1992), the solver of Sec. 5,
 * right-preconditioned with the handle's FD solve (none for IGA_PREC_NONE), one
 * right-hand side.  Device pointers rhs_dev, x_dev: N doubles; x_dev holds x0 on entry
 * when use_x0 != 0 and the solution on return.  Stops when the recursively updated
 * residual, checked after each half of an iteration (the BiCG half, then the GMRES(1)
 * half), satisfies ||r|| <= tol ||b||, or after max_iter iterations.
 *   half_steps     (out, optional) half steps taken: 2k after iteration k, 2k - 1 when
 *                  the BiCG half of iteration k met the tolerance (Sec. 5 reports
 *                  half_steps / 2 = k or k - 0.5 iterations)
 *   res_hist_host  (out, optional, host) 2 max_iter + 1 doubles: ||r|| / ||b|| before
 *                  the first step and after each half step; entries past half_steps 0
 *   true_relres    (out, optional) ||b - A_C x|| / ||b|| recomputed in FP64
 * Synchronous (waits for the handle's stream).  max_iter in 1..4096.
 * Errors: INVALID_ARG, NO_CONVERGENCE (max_iter reached with tol > 0, or a breakdown:
 * rho, (rhat, v) or (t, t) zero -- see iga_last_error), NAN, CUDA, OOM.  */
iga_status iga_solve_bicgstab(iga_handle h, const double *rhs_dev, double *x_dev, int use_x0,
                              double tol, int max_iter, int *half_steps, double *res_hist_host,
                              double *true_relres);

/* Launch shape of the Krylov reduction passes (the Arnoldi dot products and norms).
 *   IGA_GRID_LATENCY (default): about two blocks per SM, for one solve at a time;
 *   IGA_GRID_THROUGHPUT: a block per 4096 rows, at most one per SM, for many solves
 *     running at once (the batched and served forms).
 * The mode fixes the row partition of every reduction, so results are bitwise
 * reproducible among solves on handles with the same mode (alone or among others);
 * the two modes differ by rounding only.  Call it before the first solve or
 * iga_prepare; a later call drops the workspace and the captured solve graphs.
 * Must not be called while a solve is in flight on the handle.
 * Errors: INVALID_ARG (null handle, unknown mode, solve in flight). */
typedef enum { IGA_GRID_LATENCY = 0, IGA_GRID_THROUGHPUT = 1 } iga_grid_mode;
iga_status iga_set_grid_mode(iga_handle h, iga_grid_mode mode);

/* Allocate the Krylov workspace for nrhs right-hand sides and max_iter steps and
 * capture the solve graph now, so that the first solve of that size does no setup.
 * Synchronous; must not be called while a solve is in flight on the handle.  */
iga_status iga_prepare(iga_handle h, int nrhs, int max_iter);

/* FP64 throughput probe (a measurement utility; the paper has no counterpart): enqueues
 * one launch that keeps every SM's FP64 unit busy and returns the FLOPs it performs, so
 * that the caller can time it (CUDA events on `stream`) and obtain the device's FP64
 * ceiling, against which the FP64 kernels of this library are graded.
 *   kind   0: mma.sync m8n8k4 .f64 (the FP64 tensor path), 1: FP64 FMAs,
 *          2: both at once, even warps on mma.sync and odd warps on FMAs,
 *          3: both at once, every warp alternating its mma.sync and FMA chains
 *          (kinds 2 and 3 show whether the two paths share the FP64 unit)
 *   reps   1..2^24 loop turns (each launch runs for about reps x 10 us on a GB300)
 *   stream cudaStream_t (NULL = default stream); asynchronous
 *   flops  (host, may be NULL) FLOPs of the launch
 * Writes no caller memory.  Errors: INVALID_ARG, CUDA.                       */
iga_status iga_fp64_probe(int kind, int reps, void *stream, double *flops);

/* Test hook (not part of the method): writes `code` into the handle's device error word
 * -- the word a tensor-core FD kernel sets when one of its bounded waits runs out -- by a
 * host-to-device copy on the handle's stream, so that a test can check, without making
 * any device wait run out, that the next solve returns IGA_ERR_DEVICE_TIMEOUT, clears the
 * word, and that the handle stays usable.  Synchronous.  Only the tensor-core forms
 * (TF32, BF16, TF32X3, FP64_TC) have the word.  Errors: INVALID_ARG (null handle, no tensor-core FD, solve in flight), CUDA. */
iga_status iga_test_set_device_error(iga_handle h, int code);

/* Release everything the handle owns.  NULL is accepted. */
iga_status iga_destroy(iga_handle h);

/* Static English description of a status code. */
const char *iga_status_string(iga_status s);

/* Message for the last failure on the calling thread ("" if none). */
const char *iga_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IGA_FD_H */
