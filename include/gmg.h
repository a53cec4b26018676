/*
 * gmg.h - C ABI of the GB300 GMG-preconditioned FGMRES Poisson-type solver.
 *
 * Solves -div(a grad phi) = f on a uniform cell-centred 3-D grid
 * (nx x ny x nz cells on [0,lx] x [0,ly] x [0,lz]) with the 7-point
 * finite-volume discretisation of eq. (e18) (Sec. 2.2 of Lin, Zhuang, Cai,
 * Zeng, Bao, "An efficient and accurate MPI-based parallel simulator for
 * streamer discharges in three dimensions"):
 *
 *   (A phi)_p = sum_{interior faces f=(p,q)} a_f (phi_p - phi_q) / h_f^2
 *             + sum_{plate faces of p} 2 a_p (phi_p - g) / hz^2 ,
 *   a_f = (a_p + a_q) / 2  (Sec. 2.2, face means of the cell coefficient),
 *
 * Dirichlet potential g on the plates z = 0 and z = lz, zero flux through
 * the side faces x = 0, lx and y = 0, ly (the model eq. (eM), Sec. 1).  The
 * plate faces use a_f = a_p and the ghost value 2g - phi_p.
 *
 * The solver is FGMRES with right preconditioning (Algorithm 1, Sec. 3.1)
 * whose preconditioner is one geometric-multigrid V-cycle from a zero guess
 * (Sec. 3.2, eq. (eRichard), Appendix A) with an SSOR-preconditioned
 * Chebyshev smoother (eqs. (smootheq), (qntn), (e19)) and a direct solve on
 * the coarsest grid.  It stops when ||b - A phi||_2 / ||b||_2 < rtol
 * (eq. (criterion), Sec. 5.2), checked on the true FP64 residual.
 *
 * Conventions for every entry point below:
 *  - Layout: every field is a contiguous array of nz*ny*nx elements in
 *    [k][j][i] order, x fastest; cell (i,j,k) has centre
 *    ((i+1/2)hx, (j+1/2)hy, (k+1/2)hz).
 *  - Ownership: pointers named *_dev are device memory owned by the caller,
 *    read or written only during the call (the library keeps no caller
 *    pointer).  Pointers named *_host are host memory owned by the caller.
 *    The context owns all internal device workspace and frees it in
 *    gmg_destroy().
 *  - Streams: all device work is enqueued on the context's stream (given to
 *    gmg_setup / gmg_set_stream; NULL = legacy default stream).  Calls that
 *    return a result on the host (norms, solve info) synchronise that stream.
 *  - Errors: every call returns a gmg_status; nothing aborts and no C++
 *    exception crosses the ABI.  CUDA failures map to GMG_ERR_CUDA, failed
 *    device allocations to GMG_ERR_ALLOC, invalid arguments to GMG_ERR_ARG.
 *    The finest level's smoother waits for its bulk-tensor copies for about
 *    a second at most; a wait that runs out is counted on the device, and
 *    gmg_setup, gmg_update_coefficient and every solve then return
 *    GMG_ERR_CUDA (the context should be destroyed).
 *  - Threads: a context must not be used by two host threads at once.
 */
#ifndef GMG_H_
#define GMG_H_

#ifdef __cplusplus
extern "C" {
#endif

#define GMG_MAX_HISTORY 256

typedef struct gmg_ctx gmg_ctx; /* opaque: level hierarchy + Krylov workspace */

typedef enum gmg_status {
  GMG_OK = 0,
  GMG_ERR_ARG = 1,           /* invalid argument, shape or parameter        */
  GMG_ERR_CUDA = 2,          /* a CUDA runtime call failed                  */
  GMG_ERR_ALLOC = 3,         /* device memory allocation failed             */
  GMG_ERR_NOT_CONVERGED = 4, /* max_iters reached; best phi still written    */
  GMG_ERR_BREAKDOWN = 5,     /* Arnoldi/Givens breakdown that is not lucky  */
  GMG_ERR_NONFINITE = 6      /* NaN or Inf met in a norm, dot or input      */
} gmg_status;

/* Precision of the V-cycle preconditioner.  The FGMRES outer vectors, the
 * Arnoldi orthogonalisation, the Hessenberg least squares and the true
 * residual are FP64 in both modes. */
typedef enum gmg_precision { GMG_PREC_FP64 = 0, GMG_PREC_MIXED = 1 } gmg_precision;

/* Coarse-to-fine interpolation of the V-cycle (the paper's transfer figure is
 * lost).  GMG_PROLONG_OPDEP: per axis the fine child takes the parent and the
 * coarse neighbour on its side, weighted by the series conductances of the
 * fine links in between (the child sits half a fine cell from its parent's
 * centre; towards the neighbour lie the link the two coarse cells share and
 * half of the neighbour's inner link); a neighbour beyond a plate is the
 * homogeneous Dirichlet value 0, beyond a side wall it has weight 0; the
 * three axes combine as a tensor product.  With a constant coefficient it is
 * the trilinear interpolation. */
typedef enum gmg_prolongation {
  GMG_PROLONG_TRILINEAR = 0, /* cell-centred trilinear (3/4, 1/4 per axis) */
  GMG_PROLONG_CONSTANT = 1,  /* piecewise constant injection               */
  GMG_PROLONG_OPDEP = 2      /* operator-dependent weights (default)       */
} gmg_prolongation;

/* Coarse-grid operators (Sec. 3.2 is silent on them).  Both keep a 7-point
 * operator on every level.  GMG_COARSEN_SERIES gives each coarse face its own
 * coefficient: along the face normal the three fine links between the two
 * coarse cell centres (half of each coarse cell's inner link and the link
 * they share) add in series, across it the four fine columns that cross the
 * face add in parallel (their mean); a plate face takes half the inner link
 * of its coarse cell in series with the fine plate face.  A constant
 * coefficient gives the re-discretised operator.  GMG_COARSEN_MEAN
 * re-discretises eq. (e18) with the 8-child mean of the cell coefficient. */
typedef enum gmg_coarsening {
  GMG_COARSEN_MEAN = 0,      /* cell coefficient = 8-child mean             */
  GMG_COARSEN_SERIES = 1     /* per-face series-parallel coefficients
                                (default)                                   */
} gmg_coarsening;

typedef enum gmg_smoother_pc {
  GMG_PC_SGS = 0,      /* one symmetric Gauss-Seidel sweep, red-black order */
  GMG_PC_JACOBI = 1,   /* diagonal                                          */
  GMG_PC_IDENTITY = 2  /* none (plain Chebyshev)                            */
} gmg_smoother_pc;

/* Orthogonalisation of the FGMRES Arnoldi process and of the FP64 eigen-bound
 * Arnoldi.  The FP32 eigen-bound Arnoldi of the mixed set-up always takes a
 * single classical pass (the bounds only steer the FP32 smoother).  MGS runs
 * one fused pass per basis vector (about 2 FMA and 32 bytes per element per
 * vector); CGS2 runs three fused passes (about 4 FMA per element per vector),
 * which on GB300's 1/64-rate FP64 pipe is the slower of the two. */
typedef enum gmg_orthogonalization {
  GMG_ORTH_CGS2 = 0, /* classical Gram-Schmidt applied twice, fused passes */
  GMG_ORTH_MGS = 1   /* modified Gram-Schmidt as printed in Algorithm 1
                        (default)                                          */
} gmg_orthogonalization;

/* Arithmetic of the FGMRES matrix-vector product w = A z_j when z_j is the
 * FP32 V-cycle output (GMG_PREC_MIXED).  w, a and all Krylov vectors stay
 * FP64 in memory either way.  GB300 runs FP64 instructions at 1/64 of the FP32
 * rate, so the default evaluates the stencil in double-float arithmetic
 * (pairs of FP32 numbers with error-free sums and products, a 48-bit
 * significand, about 1e-14 relative to an FP64 evaluation). */
typedef enum gmg_outer_arith {
  GMG_OUTER_FP64 = 0,        /* native FP64 instructions                     */
  GMG_OUTER_DOUBLE_FLOAT = 1 /* FP32 pairs (default)                         */
} gmg_outer_arith;

/* Multigrid cycle used as the FGMRES preconditioner (Sec. 3.2).  The paper
 * preconditions the first time step, which has no previous potential and so
 * starts from a zero guess, with full multigrid, and later steps with
 * V-cycles. */
typedef enum gmg_cycle {
  GMG_CYCLE_V = 0,    /* one V-cycle from a zero guess (default)             */
  GMG_CYCLE_FMG = 1,  /* full multigrid: the right-hand side is restricted to
                         every level, the coarsest grid solved directly, and
                         each finer level takes one V-cycle from the prolonged
                         coarser result                                     */
  GMG_CYCLE_AUTO = 2  /* FMG when the solve's initial guess is zero, else V  */
} gmg_cycle;

/* Krylov method of gmg_krylov_solve: the paper's solver and the other
 * multigrid-preconditioned methods of its comparison (Sec. 5.4, Tables t1
 * and t2), all right-preconditioned with the same cycle. */
typedef enum gmg_krylov {
  GMG_KRYLOV_FGMRES = 0,   /* Algorithm 1 (fgmres_solve)                      */
  GMG_KRYLOV_GMRES = 1,    /* restarted GMRES, stores only V, x += M (V y)    */
  GMG_KRYLOV_CG = 2,       /* preconditioned conjugate gradients             */
  GMG_KRYLOV_FCG = 3,      /* flexible CG with one stored direction          */
  GMG_KRYLOV_CGS = 4,      /* conjugate gradient squared                     */
  GMG_KRYLOV_BICGSTAB = 5  /* BiCGSTAB                                       */
} gmg_krylov;

typedef struct gmg_params {
  int nx, ny, nz;              /* cells; halving all three must reach a grid
                                  whose smallest side equals coarse_min      */
  double lx, ly, lz;           /* domain lengths (> 0)                       */
  double phi_bottom, phi_top;  /* Dirichlet data on z = 0 and z = lz         */
  int coarse_min;              /* smallest side of the coarsest grid (>= 1)  */
  int cheb_steps;              /* Chebyshev steps per smoothing, 1..8        */
  int restart;                 /* FGMRES restart length m, 1..64             */
  int max_iters;               /* cap on total FGMRES iterations (>= 1)      */
  double rtol;                 /* relative residual tolerance (> 0)          */
  int eig_steps;               /* Arnoldi steps for the eigen bounds, 1..32  */
  double eig_hi, eig_lo;       /* lambda_max = eig_hi * lam_hat,
                                  lambda*    = eig_lo * lam_hat             */
  int precision;               /* gmg_precision                              */
  int prolongation;            /* gmg_prolongation                           */
  int smoother_pc;             /* gmg_smoother_pc                            */
  int orthogonalization;       /* gmg_orthogonalization                      */
  int outer_arith;             /* gmg_outer_arith: arithmetic of the Arnoldi
                                  product w = A z_j in GMG_PREC_MIXED        */
  int smoother_kernel;         /* 0: one fused pass per Chebyshev step where
                                  the level allows it (FP32, SGS, nx >= 32,
                                  ny >= 16, nz >= 8), on the finest level fed
                                  by bulk-tensor copies where nx % 4 == 0,
                                  nx >= 64, ny >= 26 and the arrays are
                                  16-byte aligned; 1: separate residual and
                                  half-sweep kernels everywhere; 2: the fused
                                  pass without the bulk-tensor copies        */
  int cycle;                   /* gmg_cycle                                  */
  int coarsening;              /* gmg_coarsening                             */
} gmg_params;

typedef struct gmg_solve_info {
  int iterations;              /* total FGMRES iterations (preconditioner calls) */
  int restarts;                /* completed restart cycles                      */
  int converged;               /* 1 if the true residual met rtol               */
  double true_rel_residual;    /* ||b - A phi|| / ||b|| in FP64 at return       */
  double bnorm;                /* ||b||                                         */
  int n_history;               /* entries used in res_history                   */
  double res_history[GMG_MAX_HISTORY]; /* least-squares residual / ||b|| per iteration */
  float setup_ms;              /* last set-up (gmg_setup / update) time, ms    */
  float solve_ms;              /* this solve, ms (host wall clock incl. syncs) */
  int fmg;                     /* 1 if this solve was preconditioned by FMG     */
  int precond_calls;           /* preconditioner applications in this solve     */
} gmg_solve_info;

/* Fill *p with the paper's defaults for an nx x ny x nz unit-cube grid:
 * plate data 0 / 1, coarse_min 4, 3 Chebyshev steps (a quadratic p_n, Sec.
 * 3.2), restart 20 (the paper uses 30, Sec. 3.1), rtol 1e-8 (Sec. 5.2),
 * 10 Arnoldi steps with factors 1.1 / 0.1 (Sec. 3.2), mixed precision,
 * operator-dependent prolongation, series-parallel coarse operators, SGS
 * smoother preconditioner, MGS, double-float Arnoldi product in mixed
 * precision. */
void gmg_default_params(gmg_params* p, int nx, int ny, int nz);

/* Build a context: copy the cell coefficient a (a_dev, FP64, > 0 and finite),
 * form the coarse operators (params.coarsening), the prolongation weights of
 * every level (GMG_PROLONG_OPDEP), estimate the Chebyshev
 * bounds of every smoothed level by Arnoldi on B^{-1} A_l (Sec. 3.2) and
 * factor the coarsest operator (Sec. 3.2, "sequential direct solver").
 * stream: a cudaStream_t or NULL.  On success *out owns all workspace.
 * Errors: GMG_ERR_ARG (bad params, a <= 0 or non-finite), GMG_ERR_ALLOC,
 * GMG_ERR_CUDA.  On error *out is NULL. */
gmg_status gmg_setup(const gmg_params* p, const double* a_dev, void* stream, gmg_ctx** out);

/* Renew the coefficient for a new time step (the matrix and preconditioner
 * are rebuilt each step, Sec. 3): same work as gmg_setup on the existing
 * workspace.  a_dev: FP64, nz*ny*nx. */
gmg_status gmg_update_coefficient(gmg_ctx* ctx, const double* a_dev);

/* Solve A phi = b with b = f + plate terms (or b = f if homogeneous_bc != 0,
 * the form used by the adjoint solve).  phi_dev holds the initial guess x0
 * on entry (zeros for a cold start; the previous step's phi for a warm
 * start, Sec. 3.2) and the solution on return, also when the solve did not
 * converge.  f_dev, phi_dev: FP64.  info may be NULL.
 * Returns GMG_OK, GMG_ERR_NOT_CONVERGED, GMG_ERR_NONFINITE or a CUDA error. */
gmg_status fgmres_solve(gmg_ctx* ctx, const double* f_dev, double* phi_dev, int homogeneous_bc,
                        gmg_solve_info* info);

/* Transport constants of eq. (eM) (Sec. 2.1, 5.2), in the units of the grid
 * lengths, potentials and densities (cm, V, cm^-3 in the paper). */
typedef struct gmg_transport_coef {
  double mu_e, mu_p;             /* mobilities (magnitudes used)              */
  double diff_x, diff_y, diff_z; /* electron diffusion D_e = diag(...)        */
  double ion_a, ion_b;           /* alpha(|E|) = ion_a P exp(-ion_b P / |E|)  */
  double pressure;               /* P (the paper: 5.7, 260, 760 Torr)         */
} gmg_transport_coef;

/* One explicit stage of the transport equations of eq. (eM) in the field
 * E = -grad(phi), the building block of the second-order semi-implicit step
 * eqs. (e1)-(e2) (predictor: c = tau/2, eval = base = n^n; corrector: c = tau,
 * base = n^n, eval = n^{n+1/2}):
 *   out_e = base_e + c [ div(mu_e E n_e) + div(D_e grad n_e) + alpha(|E|) mu_e |E| n_e ]
 *   out_p = base_p + c [ -div(mu_p E n_p) + alpha(|E|) mu_e |E| n_e ]
 * with n and E at the eval state.  Finite volumes on the grid of p (Sec. 2.2):
 * MUSCL face values with the Koren limiter phi(r) = max(0, min(2r, (1+2r)/3, 2)),
 * upwinded by the face velocity (-mu_e E_f for electrons, mu_p E_f for ions,
 * E_f from phi with mirror ghosts on the side walls and 2 g - phi on the plates,
 * g = p->phi_bottom / phi_top); densities take two layers of zero-flux ghosts;
 * |E| of the source is the cell-centred central difference field.  All arrays
 * FP64 device arrays of nx*ny*nz cells; out_e / out_p may be base_e / base_p
 * but not eval_e, eval_p or phi.  No context is needed.  Errors: GMG_ERR_ARG
 * (null or aliased pointers, bad grid or a plane nx*ny of 2^31 cells or more,
 * non-finite constants), GMG_ERR_CUDA. */
gmg_status transport_stage(const gmg_params* p, const double* base_e, const double* base_p,
                           const double* eval_e, const double* eval_p, const double* phi,
                           const gmg_transport_coef* tc, double c, double* out_e, double* out_p, void* stream);

/* dst[i] = src[i] rounded to FP32 (round to nearest, ties to even; overflow to
 * infinity; NaN stays NaN): the rounding the mixed-precision preconditioner
 * applies to its FP64 input v_j before the FP32 V-cycle (Sec. 3.1), done on the
 * integer pipe.  src: n FP64 device values, dst: n FP32 device values (no
 * overlap), both owned by the caller; enqueued on stream.  Errors: GMG_ERR_ARG
 * (null or identical pointers with n > 0), GMG_ERR_CUDA. */
gmg_status gmg_round_to_f32(const double* src, float* dst, size_t n, void* stream);

/* Both transport stages of one second-order semi-implicit step, eqs. (e1)-(e2),
 * in the field of one phi (phi^{n+1/2}):
 *   predictor  half = n + (tau/2) R(n),   corrector  out = n + tau R(half),
 * R the right-hand side of transport_stage.  The ionization rate
 * alpha(|E|) mu_e |E| depends on phi only: the predictor writes it to rate[] and
 * the corrector reads it there, so the result is bit-identical to the two
 * transport_stage calls.  All arrays FP64 device arrays of nx*ny*nz cells;
 * out_e / out_p may be n_e / n_p (in place); half_e, half_p and rate are
 * scratch owned by the caller and alias nothing else.  Errors: GMG_ERR_ARG
 * (null or aliased pointers, bad grid as in transport_stage, non-finite
 * constants or tau), GMG_ERR_CUDA. */
gmg_status transport_step(const gmg_params* p, const double* n_e, const double* n_p, const double* phi,
                          const gmg_transport_coef* tc, double tau, double* half_e, double* half_p, double* out_e,
                          double* out_p, double* rate, void* stream);

/* Solve like fgmres_solve with another Krylov method (gmg_krylov).  Each
 * method stops when its own residual estimate falls below rtol ||b||, then
 * checks the true residual and restarts from phi if that is not below rtol.
 * info->iterations counts the method's iterations (CGS and BiCGSTAB apply
 * the preconditioner twice per iteration: see info->precond_calls).  The
 * short-recurrence methods keep their vectors in the Krylov basis storage and
 * need restart >= 7.  Errors as fgmres_solve; GMG_ERR_ARG for an unknown
 * method; GMG_ERR_BREAKDOWN if a method breaks down before any progress. */
gmg_status gmg_krylov_solve(gmg_ctx* ctx, int method, const double* f_dev, double* phi_dev, int homogeneous_bc,
                            gmg_solve_info* info);

/* y = A x (the operator of eq. (e18) with zero Dirichlet data), FP64. */
gmg_status apply_operator(gmg_ctx* ctx, const double* x_dev, double* y_dev);

/* b = f + 2 a_p g / hz^2 on the plate layers (eq. (e18) with the ghost
 * cells of the Dirichlet plates), FP64. */
gmg_status assemble_rhs(gmg_ctx* ctx, const double* f_dev, double* b_dev);

/* E = -grad(phi) by cell-centred central differences (Sec. 2.2) with the
 * boundary ghosts (mirror on side walls, 2g - phi on plates).  ex, ey, ez:
 * device arrays of nz*ny*nx floats if out_fp32 != 0, else doubles. */
gmg_status field_from_potential(gmg_ctx* ctx, const double* phi_dev, void* ex_dev, void* ey_dev,
                                void* ez_dev, int out_fp32);

/* Gradient of a loss L(phi) with respect to the cell coefficient, given phi
 * and lambda = A^{-1} dL/dphi (the adjoint solve: fgmres_solve with
 * homogeneous_bc = 1 on dL/dphi; dL/df = lambda).  Not in the paper: it is
 * the derivative of the discrete operator of eq. (e18):
 *   dL/da_p = -1/2 sum_{interior f=(p,q)} (lam_p-lam_q)(phi_p-phi_q)/h_f^2
 *             - sum_{plate faces of p} 2 lam_p (phi_p - g)/hz^2 .
 * All arrays FP64. */
gmg_status adjoint_coefficient_grad(gmg_ctx* ctx, const double* phi_dev, const double* lambda_dev,
                                    double* dlda_dev);

/* Constants of the elliptic step of the semi-implicit scheme (Sec. 2.1). */
typedef struct gmg_density_coef {
  double tau;                  /* time step tau_n                             */
  double mu_e, mu_p;           /* electron / ion mobility (magnitudes used:
                                  the paper prints mu_e with both signs)      */
  double diff_x, diff_y, diff_z; /* electron diffusion D_e = diag(...)        */
  double e_over_eps0;          /* e / eps0 in the units of the densities,
                                  mobilities and lengths (1.809514e-6 V cm for
                                  cm^-3, cm^2/(V s) and cm)                   */
} gmg_density_coef;

/* Coefficient and right-hand side of the elliptic equation eq. (semi2) in its
 * discrete form eq. (e18) (Sec. 2.2), from the electron and ion densities at
 * t_n, divided through by eps0/e so that a = 1 in vacuum:
 *   a = 1 + (e/eps0) (tau/2) (|mu_p| n_p + |mu_e| n_e)
 *   f = (e/eps0) [n_p - n_e - (tau/2) sum_alpha D_alpha delta_alpha^2 n_e / h_alpha^2]
 * where delta_alpha^2 is the second difference along alpha with the densities'
 * homogeneous Neumann ghosts (ghost = interior cell).  The grid (nx, ny, nz,
 * lx, ly, lz) is taken from p; no context is needed, so the first time step
 * can assemble a before gmg_setup.  ne_dev, np_dev, a_dev, f_dev: FP64 device
 * arrays of nx*ny*nz cells, caller-owned; a_dev / f_dev may not alias the
 * densities.  stream: a cudaStream_t or NULL.  Errors: GMG_ERR_ARG (null
 * pointer, bad grid, tau < 0 or non-finite constants), GMG_ERR_CUDA. */
gmg_status assemble_coefficient_rhs(const gmg_params* p, const double* ne_dev, const double* np_dev,
                                    const gmg_density_coef* dc, double* a_dev, double* f_dev, void* stream);

/* End-to-end step with HOST buffers: copy a_host (may be NULL to keep the
 * current coefficient; else the set-up is renewed) and f_host to the device,
 * take the initial guess from phi0_host (NULL: zero, a cold start), solve,
 * optionally form E, and copy phi (and E) back into phi_host (and
 * ex/ey/ez_host).  ex/ey/ez_host may all be NULL (no field); they hold
 * floats if field_fp32 != 0, else doubles.  Host buffers should be pinned for
 * full copy bandwidth.  Device staging buffers are allocated on first use and
 * kept by the context.  Returns like fgmres_solve. */
gmg_status gmg_solve_host(gmg_ctx* ctx, const double* a_host, const double* f_host, const double* phi0_host,
                          double* phi_host, void* ex_host, void* ey_host, void* ez_host, int field_fp32,
                          gmg_solve_info* info);

/* gmg_solve_host, pipelined: returns once the solve has finished (info filled)
 * and the field kernel is enqueued; the copy-out of phi (and E) is held back.
 * The next host-array call enqueues it on the context's copy-out stream once
 * its own upload of a is done (the set-up waits for that upload, which so has
 * the link to itself), and it then overlaps that call's set-up and solve;
 * gmg_host_wait enqueues it if no call comes first.  phi_host and ex/ey/ez_host
 * must stay valid and unread until gmg_host_wait(ctx) returns; a_host, f_host
 * and phi0_host have been consumed only when the next call, or gmg_host_wait,
 * returns.  The next call's staging writes wait for the copy-out.  Errors
 * return like gmg_solve_host, with every copy completed. */
gmg_status gmg_solve_host_async(gmg_ctx* ctx, const double* a_host, const double* f_host, const double* phi0_host,
                                double* phi_host, void* ex_host, void* ey_host, void* ez_host, int field_fp32,
                                gmg_solve_info* info);

/* Waits for every copy and kernel of the context's host-array solves (the
 * copy-out of gmg_solve_host_async included).  Errors: GMG_ERR_ARG (null ctx),
 * GMG_ERR_CUDA (a failed copy or kernel). */
gmg_status gmg_host_wait(gmg_ctx* ctx);

gmg_status gmg_set_stream(gmg_ctx* ctx, void* stream);
void gmg_destroy(gmg_ctx* ctx);
const char* gmg_status_string(gmg_status s);

/* ---- Inspection entry points (used by the kernel-by-kernel parity tests) ----
 * Levels are numbered 0 = coarsest ... gmg_num_levels()-1 = finest.
 * "level precision" is FP32 in GMG_PREC_MIXED and FP64 in GMG_PREC_FP64. */
int gmg_num_levels(const gmg_ctx* ctx);

/* Grid size and Chebyshev bounds (lambda_max, lambda*) of a level; the
 * coarsest level reports 0 bounds (it is solved directly). */
gmg_status gmg_level_info(const gmg_ctx* ctx, int level, int* nx, int* ny, int* nz, double* lam_max,
                          double* lam_min);

/* Replace the Chebyshev bounds of level l (1 <= l < gmg_num_levels) with
 * lam_max > lam_min > 0 (both finite), until the next set-up renews them.
 * Lets a test run the smoother (Sec. 3.2, eq. (qntn)) of both sides on one
 * interval given from outside.  GMG_ERR_ARG otherwise. */
gmg_status gmg_level_set_bounds(gmg_ctx* ctx, int level, double lam_max, double lam_min);

/* Copy the FP64 cell coefficient of a level (the finest level's a, or the
 * 8-child means with GMG_COARSEN_MEAN) into out_dev (FP64, that level's
 * size).  GMG_ERR_ARG on a level that carries face coefficients. */
gmg_status gmg_level_coefficient(gmg_ctx* ctx, int level, double* out_dev);

/* The face coefficients of a level's operator, divided by h^2 (the matrix
 * entries), widened to FP64: kx_dev[k][j][i] couples cells i-1 and i (0 at
 * i = 0), ky_dev likewise along y (0 at j = 0), kz_dev[k][j][i] couples
 * k-1 and k, and at k = 0 holds the bottom plate's 2 a / hz^2-type entry;
 * ktop_dev[j][i] (ny*nx) the top plate's.  Each of kx, ky, kz has the
 * level's size.  Works on every level (cell-form levels give the face means
 * of eq. (e18)). */
gmg_status gmg_level_faces(gmg_ctx* ctx, int level, double* kx_dev, double* ky_dev, double* kz_dev,
                           double* ktop_dev);

/* One V-cycle from a zero guess, z = M v (Appendix A), or full multigrid if
 * the context's cycle is GMG_CYCLE_FMG: v_dev, z_dev FP64 of the finest size.
 * In mixed mode v is rounded to FP32 and the cycle runs in FP32; z is widened
 * back to FP64. */
gmg_status gmg_apply_preconditioner(gmg_ctx* ctx, const double* v_dev, double* z_dev);

/* w = A z for an FP32 z of the finest size, as FGMRES forms its Arnoldi
 * product in GMG_PREC_MIXED (arithmetic per params.outer_arith); w FP64.
 * GMG_ERR_ARG in GMG_PREC_FP64 mode, where z_j is FP64 (use apply_operator). */
gmg_status gmg_apply_outer(gmg_ctx* ctx, const float* z_dev, double* w_dev);

/* y = A_l x on a level, in level precision (x_dev, y_dev of that type). */
gmg_status gmg_level_apply(gmg_ctx* ctx, int level, const void* x_dev, void* y_dev);

/* cheb_steps preconditioned Chebyshev steps on level l (l >= 1) for
 * A_l x = b, in level precision; x_is_zero != 0 ignores x_dev's contents
 * (the pre-smoothing from a zero guess). */
gmg_status gmg_level_smooth(gmg_ctx* ctx, int level, const void* b_dev, void* x_dev, int x_is_zero);

/* z = B^{-1} r for the smoother preconditioner on level l, level precision. */
gmg_status gmg_level_smoother_pc(gmg_ctx* ctx, int level, const void* r_dev, void* z_dev);

/* coarse_dev = mean of 8 children of (b - A_l x) on level l (the fused
 * residual + restriction); level precision; coarse_dev has level l-1's size. */
gmg_status gmg_level_residual_restrict(gmg_ctx* ctx, int level, const void* b_dev, const void* x_dev,
                                       void* coarse_dev);

/* x_l += P e (prolongation from level l-1, then correction), level precision. */
gmg_status gmg_level_prolong_add(gmg_ctx* ctx, int level, const void* e_dev, void* x_dev);

/* x = A_0^{-1} b on the coarsest level (direct solve), level precision. */
gmg_status gmg_coarse_solve(gmg_ctx* ctx, const void* b_dev, void* x_dev);

/* Largest real part of the eigenvalues of an m x m upper Hessenberg matrix
 * (row-major, m <= 64), by Francis double-shift QR on the host; used for
 * lam_hat of the eigen bounds (Sec. 3.2).  Host memory only; needs no GPU.
 * Returns GMG_ERR_ARG for m out of range, GMG_ERR_BREAKDOWN if QR fails to
 * converge. */
gmg_status gmg_hessenberg_max_real_eig(const double* h_host, int m, double* out);

/* ---- Per-kernel profile (tracing) ----
 * Launch counts are always kept.  With profiling enabled, every kernel launch
 * is bracketed by CUDA events on the context's stream, and each launch's
 * algorithmic bytes (every array the kernel must touch, read or written
 * once) are accumulated per kernel class.  Timing adds two event records per
 * launch and no synchronisation beyond the solver's own.  Launches that move
 * fewer algorithmic bytes than gmg_profile_min_bytes (default 0) are counted
 * but not timed, which keeps the host from falling behind the GPU on the
 * coarse levels' many small launches. */
gmg_status gmg_profile_enable(gmg_ctx* ctx, int on);
gmg_status gmg_profile_min_bytes(gmg_ctx* ctx, double min_bytes);
gmg_status gmg_profile_reset(gmg_ctx* ctx);
int gmg_profile_num_kernels(void);
/* Totals of kernel class k (0 <= k < gmg_profile_num_kernels()): its name
 * (static string), launches, launches timed, summed event time in ms and
 * summed algorithmic bytes of the timed launches.  Synchronises the stream. */
gmg_status gmg_profile_get(gmg_ctx* ctx, int k, const char** name, long long* launches,
                           long long* timed_launches, double* total_ms, double* total_bytes);

/* ---- Coarsest-grid direct solve without allocation ----
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (device memory wholly reserved by a
 * framework's pool, real-time loops that must not take cudaMalloc's implicit
 * device synchronisation or out-of-memory failure, code under a fixed memory
 * budget).  It does what gmg_setup does for the coarsest grid and what
 * gmg_coarse_solve then applies, in FP64: assemble the dense operator of the
 * grid described by p (nx, ny, nz, lx, ly, lz; other fields ignored) from the
 * cell coefficient a_dev, factor it (Cholesky), and write x = A^{-1} b.
 * a_dev, b_dev, x_dev: FP64 device arrays of nx*ny*nz elements, caller-owned;
 * stream: cudaStream_t or NULL.
 * Scratch: one file-scope __device__ array sized for
 * GMG_NOALLOC_MAX_UNKNOWNS unknowns (about 6 MB), held by every GPU that
 * loads the library until the process exits; the call makes no device or
 * pinned-host allocation.  Each call looks up the array's address on the
 * current device (cudaGetSymbolAddress), so it is valid on any device and
 * after a device reset.  Every call overwrites the whole array; calls that
 * overlap on the GPU race on it.
 * Errors: GMG_ERR_ARG if nx*ny*nz > GMG_NOALLOC_MAX_UNKNOWNS or an argument is
 * invalid (a side below 1, a length not positive or not finite), GMG_ERR_BREAKDOWN if the operator is not positive definite,
 * GMG_ERR_CUDA.  Synchronises the stream once (to read the factorisation
 * status). */
#define GMG_NOALLOC_MAX_UNKNOWNS 512
gmg_status gmg_coarse_solve_noalloc(const gmg_params* p, const double* a_dev, const double* b_dev,
                                    double* x_dev, void* stream);

/* Test hook: make the n-th next device allocation of the library fail
 * (n >= 1), as if the device were out of memory; n = 0 disables it.  Lets
 * the host-side error paths be tested without exhausting a shared GPU. */
void gmg_test_fail_allocation_after(int n);

#ifdef __cplusplus
}
#endif

#endif /* GMG_H_ */
