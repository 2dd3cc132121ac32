/*
 * sipg.h -- C ABI of the GB300 matrix-free SIPG library (libsipg.so).
 *
 * Method: Krank, Fehn, Wall, Kronbichler, "A high-order semi-explicit
 * discontinuous Galerkin solver for 3D incompressible flow with application to
 * DNS and LES of turbulent channel flow" (arXiv:1607.01323).  The library
 * evaluates, matrix-free and by sum factorisation (Sec. 5), the symmetric
 * interior-penalty operators that the paper's conjugate-gradient solvers apply
 * at every iteration (Sec. 5.1):
 *   - the pressure Poisson operator L of Sec. 3.2 (ii) (fluxes P*, Pi*,
 *     penalty of Eq. (taue) with the max rule of Eq. (tau)), Eq. (poissonmat);
 *   - the viscous Helmholtz operator (gamma0/dt) M - F^nu of Eq. (viscous), in
 *     Laplace form (gamma0/dt) M + nu L per velocity component;
 *   - the tensorial inverse mass matrix (Sec. 5);
 * plus the Jacobi / inverse-mass / FP32-Chebyshev preconditioned CG of
 * Sec. 5.1 and an adjoint gradient with respect to a per-cell viscosity.
 *
 * Discretisation: Q_k on hexahedra with nodal Lagrange polynomials on the
 * Gauss-Lobatto points (Sec. 3.1), Gauss quadrature with k+1 points per
 * direction (Sec. 5), iso-parametric degree-k mapping (Sec. 5).  Meshes are
 * structured boxes of nx x ny x nz cells whose map is separable per direction:
 * affine, or affine in x and z with the tanh wall-normal grading of Sec. 7.1.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status (sipg_status) and never aborts,
 *     traps or exits; sipg_last_error() returns a thread-local message for the
 *     last failure on the calling thread.
 *   - Host arguments are validated before any work: NULL pointers, ranges,
 *     sizes.  CUDA errors map to SIPG_ECUDA.
 *   - Vector layout: x[comp][cell][c][b][a], a along x fastest, cells
 *     numbered cell = (iz * ny + iy) * nx + ix; n_dofs = ncell * (k+1)^3 per
 *     component.  Vectors are contiguous DEVICE pointers owned by the caller,
 *     on the device that was current when the mesh was created; the library
 *     never frees them.  x and y must not overlap.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  The apply
 *     entry points are asynchronous on that stream; sipg_cg_solve returns
 *     after the solve has finished (it reads convergence data to the host).
 *   - A sipg_mesh is not thread-safe: do not use one mesh from two host
 *     threads at the same time.
 */
#ifndef SIPG_H
#define SIPG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sipg_mesh sipg_mesh; /* opaque, owned by the library */

typedef enum {
  SIPG_OK = 0,
  SIPG_MAXITER = 1,       /* solver stopped at maxit without reaching rtol     */
  SIPG_EINVAL = -1,       /* invalid argument (see sipg_last_error)             */
  SIPG_ECUDA = -2,        /* a CUDA runtime call failed                        */
  SIPG_ENOMEM = -3,       /* device or host allocation failed                  */
  SIPG_BREAKDOWN = -4,    /* CG breakdown: p^T A p <= 0 or not finite          */
  SIPG_NONFINITE = -5     /* right-hand side or residual not finite            */
} sipg_status;

typedef enum { SIPG_BC_PERIODIC = 0, SIPG_BC_DIRICHLET = 1, SIPG_BC_NEUMANN = 2 } sipg_bc;
typedef enum {
  SIPG_MAP_AFFINE = 0,
  SIPG_MAP_CHANNEL_TANH = 1,
  SIPG_MAP_CHANNEL_LINEAR = 2,
  SIPG_MAP_PERTURBED = 3
} sipg_map;
/* SIPG_OP_VISCOUS: mass_coef M + the divergence-form viscous operator of
 * sipg_apply_viscous_f64 (3 coupled components; CG with SIPG_PC_NONE or
 * SIPG_PC_INVMASS). */
typedef enum { SIPG_OP_LAPLACE = 0, SIPG_OP_HELMHOLTZ = 1, SIPG_OP_VISCOUS = 2 } sipg_op;
typedef enum { SIPG_F64_NATIVE = 0, SIPG_F64_DOUBLE_FLOAT = 1 } sipg_f64_arith;
typedef enum {
  SIPG_PC_NONE = 0,
  SIPG_PC_JACOBI = 1,     /* z = diag(A)^-1 r (Sec. 5.1: the diagonal computed once)   */
  SIPG_PC_INVMASS = 2,    /* z = M^-1 r (Sec. 5.1: viscous solver preconditioner)       */
  SIPG_PC_CHEB_F32 = 3,   /* Chebyshev in FP32 with the FP32 operator (Sec. 5.1)         */
  SIPG_PC_GMG_F32 = 4     /* one geometric-multigrid V-cycle in FP32 (Sec. 5.1)         */
} sipg_precond;

/* Mesh description.  "Dirichlet" is the side where the unknown is prescribed
 * (homogeneous data): the SIPG boundary terms with penalty 2 tau (Sec. 3.2 (ii),
 * pressure on dOmega^N; Sec. 3.2 (iii), velocity on dOmega^D).  "Neumann" sides
 * carry no operator term.  Periodic sides must be paired (lo and hi) and are
 * treated as interior faces.  map = SIPG_MAP_CHANNEL_TANH maps the global
 * wall-normal coordinate eta in [0,1] to
 *   y = lo[1] + (hi[1]-lo[1]) (1 + tanh(gamma (2 eta - 1)) / tanh(gamma)) / 2
 * (Sec. 7.1 with delta = 1 for lo=-1, hi=1); x and z stay affine.
 * map = SIPG_MAP_CHANNEL_LINEAR takes the same y at the cell boundaries
 * eta_j = j / n[1] and is affine inside each cell (straight cells on the
 * graded vertices; the coarse levels of the multigrid hierarchy).
 * map = SIPG_MAP_PERTURBED is the box plus a smooth displacement that vanishes
 * on the box boundary (general, non-separable metrics):
 *   x_i += amplitude (hi_i - lo_i) c_i b(s) cos(pi (s_(i+1) - s_(i+2))),
 *   b(s) = sin(pi s_x) sin(pi s_y) sin(pi s_z), s the global reference
 *   coordinate in [0,1]^3, c_i = 2 f_i / 65535 - 1 with f_i the 16-bit field
 *   i of seed.
 * Its geometry is stored per quadrature point (56 B per DoF plus face data);
 * it supports the FP64 Laplace / Helmholtz / mass applies and the diagonal
 * with a constant viscosity, and sipg_cg_solve with SIPG_PC_NONE or
 * SIPG_PC_JACOBI; the other entry points need a separable map and return
 * SIPG_EINVAL. */
typedef struct {
  int n[3];          /* cells per direction, each >= 1                         */
  double lo[3];      /* box corner                                             */
  double hi[3];      /* box corner, hi > lo                                    */
  int bc_lo[3];      /* sipg_bc per side                                       */
  int bc_hi[3];
  int map;           /* sipg_map                                               */
  double gamma;      /* grading parameter (> 0) for SIPG_MAP_CHANNEL_TANH       */
  double amplitude;  /* SIPG_MAP_PERTURBED: displacement size (>= 0)          */
  unsigned long long seed; /* SIPG_MAP_PERTURBED: displacement coefficients  */
} sipg_mesh_desc;

/* Create a mesh on the current CUDA device.  The degree defaults to k = 3 and
 * the penalty factor to 1; geometry tables are built on the device.
 * Errors: EINVAL (bad description, unpaired periodic sides), ENOMEM, ECUDA. */
int sipg_create_mesh(const sipg_mesh_desc* desc, sipg_mesh** out);

/* Free the mesh and its device tables.  NULL is accepted.  Synchronises the
 * device first so that no launch still reads the tables. */
int sipg_destroy_mesh(sipg_mesh* mesh);

/* Polynomial degree 1 <= k <= 7 of the nodal GLL basis (Sec. 3.1); rebuilds
 * the 1D tables: Gauss rule with k+1 points (Sec. 5), iso-parametric
 * degree-k interpolation of the map (Sec. 5), per-layer mass / stiffness /
 * inverse-mass matrices, face derivative vectors and penalty terms. */
int sipg_set_degree(sipg_mesh* mesh, int k);

/* tau = factor * tau_IP of Eq. (taue) (factor > 0; default 1).  factor = 1/3
 * gives (k+1)^2/h on interior cubes. */
int sipg_set_penalty(sipg_mesh* mesh, double factor);

/* Scalar DoFs per component: ncell * (k+1)^3 (host output). */
int sipg_n_dofs(const sipg_mesh* mesh, long long* n);

/* Number of cells (host output). */
int sipg_n_cells(const sipg_mesh* mesh, long long* n);

/* Physical coordinates of the nodal points: xyz[3 * i + d] for DoF i of one
 * component (HOST buffer of 3 * n_dofs doubles, caller-owned). */
int sipg_node_coordinates(const sipg_mesh* mesh, double* xyz_host);

/* Per-cell penalty tau_e of Eq. (taue) times the penalty factor (HOST buffer of
 * ncell doubles, caller-owned). */
int sipg_penalty_values(const sipg_mesh* mesh, double* tau_host);

/* y = L x: the SIPG Laplacian of Sec. 3.2 (ii) / Eq. (poissonmat), applied to
 * ncomp >= 1 independent components (Sec. 5, sum factorisation). */
int sipg_apply_laplace_f64(const sipg_mesh* mesh, const double* x, double* y, int ncomp, void* stream);
int sipg_apply_laplace_f32(const sipg_mesh* mesh, const float* x, float* y, int ncomp, void* stream);

/* y = mass_coef M x + nu L x, the viscous operator of Eq. (viscous) in
 * Laplace form (mass_coef = gamma0/dt >= 0).  If nu_cell (DEVICE, ncell
 * values > 0) is not NULL it replaces nu cell by cell: consistency terms use
 * the average of nu grad u, the penalty max(nu-, nu+) (the paper has constant
 * nu only). */
int sipg_apply_helmholtz_f64(const sipg_mesh* mesh, double mass_coef, double nu, const double* nu_cell,
                             const double* x, double* y, int ncomp, void* stream);
int sipg_apply_helmholtz_f32(const sipg_mesh* mesh, float mass_coef, float nu, const float* nu_cell,
                             const float* x, float* y, int ncomp, void* stream);

/* y = M x, the block-diagonal mass matrix with the Gauss (k+1) rule (Sec. 4.4). */
int sipg_apply_mass_f64(const sipg_mesh* mesh, const double* x, double* y, int ncomp, void* stream);

/* y = M^-1 x, the tensorial inverse mass matrix of Sec. 5: with n_q = k+1 the
 * 1D node-to-quadrature matrices are square and are inverted individually. */
int sipg_apply_inverse_mass_f64(const sipg_mesh* mesh, const double* x, double* y, int ncomp, void* stream);

/* diag(A) for op = SIPG_OP_LAPLACE (mass_coef, nu, nu_cell ignored) or
 * SIPG_OP_HELMHOLTZ; diag is a DEVICE buffer of n_dofs doubles (one component).
 * Sec. 5.1: the matrix diagonal used by Jacobi and Chebyshev. */
int sipg_diagonal_f64(const sipg_mesh* mesh, int op, double mass_coef, double nu, const double* nu_cell,
                      double* diag, void* stream);

/* Options of sipg_cg_solve. */
typedef struct {
  int op;                 /* sipg_op                                                       */
  double mass_coef;       /* Helmholtz: gamma0/dt                                          */
  double nu;              /* Helmholtz: viscosity (ignored when nu_cell != NULL)           */
  const double* nu_cell;  /* Helmholtz: DEVICE [ncell] or NULL                              */
  int precond;            /* sipg_precond                                                  */
  int cheb_degree;        /* Chebyshev steps (>= 1); degree d uses d-1 operator products   */
  double cheb_range;      /* lambda_min = lambda_max / cheb_range (> 1)                     */
  double cheb_lmax;       /* > 0: use this lambda_max of D^-1 A; <= 0: estimate (Lanczos)   */
  int cheb_lanczos_steps; /* CG steps of the estimate (>= 2)                                */
  int zero_mean;          /* project b and every A p onto zero mean (Sec. 5.1)              */
  double rtol;            /* stop when ||r||_2 <= rtol ||b||_2 (recursive residual)        */
  int maxit;              /* >= 1                                                          */
  int flexible;           /* Polak-Ribiere beta (always used with SIPG_PC_CHEB_F32)         */
  int use_graph;          /* capture check_every iterations in one CUDA graph and replay it  */
  int check_every;        /* iterations between host convergence checks (>= 1)             */
  /* SIPG_PC_GMG_F32 (Laplace, one component): */
  int mg_degree;          /* Chebyshev smoother steps before and after the coarse correction */
  double mg_range;        /* smoothing range: [lambda_max / mg_range, lambda_max] per level   */
  double mg_coarse_tol;   /* coarse Chebyshev: degree where the error estimate reaches this   */
  int mg_coarse_maxdeg;   /* upper bound on that degree                                       */
} sipg_cg_opts;

/* Fill opts with defaults: Laplace, Jacobi, rtol 1e-10, maxit 10000, Chebyshev
 * degree 4, range 20, estimated lambda_max with 20 steps, graph on, checks
 * every 16 iterations; multigrid smoother degree 5, range 20, coarse
 * tolerance 1e-3 (Sec. 5.1), coarse degree at most 200. */
int sipg_cg_default_opts(sipg_cg_opts* opts);

/* Solve A x = b by preconditioned CG (Sec. 5.1) with the matrix-free FP64
 * operator.  b, x: DEVICE, ncomp * n_dofs doubles; x holds the initial guess
 * on entry and the solution on return.  The ncomp components form one
 * block-diagonal system (one CG, inner products over all components).
 * iters_out / relres_out (HOST, may be NULL) receive the iteration count and
 * ||r||/||b|| of the recursive residual.  Synchronous.  Returns SIPG_OK,
 * SIPG_MAXITER, SIPG_BREAKDOWN, SIPG_NONFINITE or an error.  Workspace
 * (5 vectors, plus 5 FP32 vectors for SIPG_PC_CHEB_F32) is allocated by the
 * library and cached on the mesh. */
int sipg_cg_solve(sipg_mesh* mesh, const sipg_cg_opts* opts, const double* b, double* x, int ncomp,
                  void* stream, int* iters_out, double* relres_out);

/* Allocation-free variant of sipg_cg_solve.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- for
 * example a host application whose device memory is owned by its own pool or
 * caching allocator (a cudaMalloc outside that pool can fail or fragment it),
 * a deployment with a fixed device-memory budget accounted for up front, or a
 * latency-critical loop that cannot afford the implicit device
 * synchronisation of cudaMalloc / cudaFree.
 *
 * The caller still passes b and x (DEVICE, as for sipg_cg_solve).  The solver's
 * workspace (5 vectors, the diagonal, partial sums, the solver record) comes
 * from one file-scope __device__ array of 16 MiB inside libsipg.  A GPU holds
 * those 16 MiB from the moment the library's CG module is loaded on it until
 * the process exits; with CUDA's lazy module loading (the default) that load
 * can be the first call of this function, which then makes a driver-side
 * reservation, so make one warm-up call outside any stream capture and any
 * allocation-sensitive region.  The array bounds the problem to about 348,000
 * unknowns (ncomp * n_dofs); larger problems are rejected with SIPG_EINVAL and
 * a message giving the bytes needed.  The function calls no cudaMalloc,
 * cudaFree or other allocating routine, creates no stream, event or graph,
 * and runs on `stream` directly; it is synchronous like sipg_cg_solve.  In
 * double-float arithmetic it uses the mesh's scale word, which
 * sipg_create_mesh allocated.  Preconditioners: SIPG_PC_NONE, SIPG_PC_JACOBI,
 * SIPG_PC_INVMASS (SIPG_PC_CHEB_F32 needs FP32 buffers and is rejected);
 * use_graph is ignored, no per-apply timing is recorded, and the mesh's
 * profiling setting is left as it is.
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress, with
 * the mesh's device current), so the address stays right across a
 * cudaDeviceReset.  Every call shares the array and it keeps the previous
 * call's contents (the solver clears what must start from zero), so calls
 * that overlap on the GPU -- on two streams, two host threads or two meshes at
 * once -- race on the array and must be serialised by the caller.  Returns the
 * same statuses as sipg_cg_solve. */
int sipg_cg_solve_noalloc(sipg_mesh* mesh, const sipg_cg_opts* opts, const double* b, double* x, int ncomp,
                          void* stream, int* iters_out, double* relres_out);

/* Geometric multigrid (Sec. 5.1), the preconditioner SIPG_PC_GMG_F32.
 *
 * Levels: the mesh, then the mesh with half the cells in every direction whose
 * count is even and > 1, and so on down to the level where no direction can be
 * halved (one cell for power-of-two meshes).  Every level keeps the degree,
 * penalty factor and boundary conditions and re-discretises the SIPG Laplacian
 * on its own geometry tables; on the coarse levels of a tanh channel each cell
 * is straight between the graded vertices (SIPG_MAP_CHANNEL_LINEAR).
 * One V-cycle, entirely in FP32 with the FP32 operator: on each level
 * mg_degree Chebyshev steps on D^-1 A from zero (D = diag(A) of the level,
 * interval [lambda_max / mg_range, lambda_max]), the residual restricted to the
 * next level, the coarse correction prolongated and added, and mg_degree
 * Chebyshev steps from that iterate; on the coarsest level a Chebyshev
 * iteration from zero on [lambda_min, lambda_max] whose degree is the smallest
 * with 2 s^d / (1 + s^2d) <= mg_coarse_tol, s = (sqrt(kappa) - 1) / (sqrt(kappa) + 1).
 * Prolongation evaluates the parent cell's polynomial at the child's nodes
 * (tensorial embedding); restriction is its transpose.  The eigenvalue
 * estimates come from cheb_lanczos_steps Jacobi-PCG steps on each level
 * (Lanczos), lambda_max with a factor 1.1; on the coarsest level up to 120
 * steps give lambda_min (factor 0.9) and lambda_max (factor 1.1).  No
 * zero-mean projection inside the cycle (Sec. 5.1).
 *
 * sipg_mg_setup builds the levels and the estimates for the options' mg_*
 * fields and cheb_lanczos_steps (op must be SIPG_OP_LAPLACE); the result is
 * cached on the mesh and reused by every later sipg_cg_solve with
 * SIPG_PC_GMG_F32 and the same options (sipg_cg_solve sets it up on first use;
 * sipg_set_degree and sipg_set_penalty drop it).  Synchronous.  Device memory:
 * six FP32 vectors per level plus two FP64 vectors of the finest size. */
int sipg_mg_setup(sipg_mesh* mesh, const sipg_cg_opts* opts, void* stream);

/* The hierarchy built by sipg_mg_setup (HOST outputs, arrays of max_levels
 * entries, NULL allowed): number of levels, cells per direction of each level
 * (n_cells[3 * l + d]), the lambda_max used on each level (for the coarsest,
 * the upper end of its interval), the coarse interval's lower end and the
 * coarse Chebyshev degree.  EINVAL if no hierarchy is set up. */
int sipg_mg_info(const sipg_mesh* mesh, int max_levels, int* nlevels, int* n_cells, double* lmax,
                 double* coarse_lmin, int* coarse_degree);

/* z = V(r): one V-cycle of the hierarchy set up on the mesh, applied to the
 * FP64 vector r (DEVICE, n_dofs doubles; rounded to FP32), result z (DEVICE,
 * n_dofs doubles).  Asynchronous on `stream`. */
int sipg_mg_vcycle(sipg_mesh* mesh, const double* r, double* z, void* stream);

/* ---------------------------------------------------------------------------
 * Pressure-projection operators of the dual-splitting scheme, variant V3c
 * (Sec. 3.3).  Velocities are 3 components u[d][cell][c][b][a] (d = x, y, z),
 * pressures 1 component; DEVICE pointers, FP64, asynchronous on `stream`.
 * The paper's factors gamma0/dt and dt/gamma0 are left to the caller.
 * {{w}}^ND (Sec. 3.1) is the average on interior and periodic faces and the
 * own trace on every boundary face (Dirichlet and Neumann sides alike). */

/* y = D u, Eq. (av3): y_i = (grad phi_i, u)_e - (phi_i, {{u}}^ND . n)_de
 * (u: 3 * n_dofs, y: n_dofs). */
int sipg_apply_divergence_f64(const sipg_mesh* mesh, const double* u, double* y, void* stream);

/* y = G p, Eq. (bv3): y_(d,i) = (d phi_i / d x_d, p)_e - (phi_i, {{p}}^ND n_d)_de
 * (p: n_dofs, y: 3 * n_dofs).  On periodic faces G = -D^T. */
int sipg_apply_gradient_f64(const sipg_mesh* mesh, const double* p, double* y, void* stream);

/* tau[e] = zeta * |ubar_e| * V_e^(1/3) * dt, Eq. (tauD), with ubar_e the
 * volume-averaged velocity of cell e (u: 3 * n_dofs; tau: ncell). */
int sipg_tau_div_f64(const sipg_mesh* mesh, const double* u, double zeta, double dt, double* tau, void* stream);

/* y = (M + tau_e B) u cell by cell, the operator of Eq. (div-div):
 * B_(d,d') = (d phi_i / d x_d, d phi_j / d x_d')_e; tau: ncell values >= 0. */
int sipg_apply_divdiv_f64(const sipg_mesh* mesh, const double* tau, const double* u, double* y, void* stream);

/* Solve (M + tau_e B) x = rhs on every cell independently (the local
 * projection of Eq. (div-div)) by CG preconditioned with the inverse of the
 * component-diagonal blocks, (M_d + tau_e K_d)^-1 along d and the 1D inverse
 * mass along the other directions (exact tensor products; the tensorial
 * M^-1 when tau_e = 0), one thread block per cell; x holds the initial guess
 * on entry.  A cell stops when ||r|| <= rtol ||rhs_e|| or after maxit
 * iterations.  Synchronous.  iters_out (HOST, may be NULL) receives the
 * largest iteration count over the cells.  Returns SIPG_MAXITER if a cell did
 * not converge, SIPG_BREAKDOWN on a non-positive curvature. */
int sipg_project_divdiv_f64(sipg_mesh* mesh, const double* tau, const double* rhs, double* x, double rtol,
                            int maxit, void* stream, int* iters_out);

/* y = mass_coef M u + A_nu u, the viscous operator of the implicit viscous
 * step in the paper's divergence form (Sec. 3.2 (iii)): A_nu from
 * (eps(v), 2 nu eps(u))_e with the symmetric interior-penalty fluxes U* and
 * F^nu* (penalty tau of Eq. (taue) / Eq. (tau)), homogeneous boundary data;
 * the three velocity components are coupled.  u, y: DEVICE, 3 * n_dofs doubles
 * (components x, y, z).  Computed as mass_coef M u + nu L u (the SIPG
 * Laplacian per component, in the mesh's FP64 arithmetic) plus nu T u, the
 * transposed-gradient coupling (FP64).  On coarse curved meshes the form may
 * need a penalty factor above 1 to stay definite (4 wall-normal layers of the
 * tanh channel at k = 2 need 2). */
int sipg_apply_viscous_f64(const sipg_mesh* mesh, double mass_coef, double nu, const double* u, double* y,
                           void* stream);

/* y = the convective term of the explicit convective step, Eq. (convstepspat):
 * y_(i,a) = (grad phi_a, u_i u)_e - (phi_a, (F^c* n)_i)_de summed over the
 * cells, with F^c(u) = u (x) u and the local Lax-Friedrichs flux (Sec. 3.2
 * (i)): {{u (x) u}} n + Lambda/2 (u^- - u^+) on interior and periodic faces,
 * Lambda = max(2|u^- . n|, 2|u^+ . n|) per quadrature point; u^- (u^- . n)
 * + Lambda u^- on no-slip (Dirichlet, g = 0) faces; u^- (u^- . n) on Neumann
 * faces.  Cell and face integrals use floor(3k/2) + 1 Gauss points per
 * direction (Sec. 5, over-integration).  u, y: DEVICE, 3 * n_dofs doubles
 * (components x, y, z), must not overlap; y is overwritten.  Evaluated in the
 * mesh's FP64 arithmetic (sipg_set_f64_arithmetic).  Nonlinear in u: the
 * result is not M^-1-scaled (apply sipg_apply_inverse_mass_f64 with ncomp = 3 for
 * the explicit update). */
int sipg_apply_convective_f64(const sipg_mesh* mesh, const double* u, double* y, void* stream);

/* ------------------------------------------------------------------------
 * The dual-splitting time step (Sec. 2.2) with the spatial variant V3c.
 *
 * One step from t^n to t^(n+1) = t^n + dt with the order-J BDF / extrapolation
 * pair (gamma0, alpha_i, beta_i of Karniadakis, Israeli and Orszag 1991):
 *  (i)   M u_hat = (M sum alpha_i u^(n-i) + dt sum beta_i C(u^(n-i)) + dt M f) / gamma0,
 *        C the convective term of sipg_apply_convective_f64, f a constant body
 *        force (Eq. (convstepspat));
 *  (ii)  L_N p = (gamma0/dt) D u_hat + (q, h)_walls with D of Eq. (av3), L_N the
 *        SIPG Laplacian with Neumann data on the no-slip walls, and
 *        h = -(sum beta_i (div F^c(u^(n-i)) + nu curl omega^(n-i)) - f) . n, the
 *        flux Pi* of Eq. (ipflux) (omega the cell-wise L2 projection of curl u,
 *        evaluated from the wall cell at the k+1 Gauss points of each wall
 *        face); solved for the zero-mean p by CG (Jacobi or the FP32 multigrid
 *        V-cycle);
 *  (iii) (M + tau_D B) u_hathat = M u_hat + (dt/gamma0) G p, Eq. (div-div) with G
 *        of Eq. (bv3) and tau_D of Eq. (tauD) from u^n (per-cell CG);
 *  (iv)  ((gamma0/dt) M + A_nu) u^(n+1) = (gamma0/dt) M u_hathat with the
 *        divergence-form viscous operator (M^-1-preconditioned CG).
 * The pressure and viscous CG start from the order-J extrapolations
 * sum beta_i p^(n-i) and sum beta_i u^(n-i) (Sec. 5.1), so that low relative
 * tolerances still give accurate solutions.
 * Velocity boundaries: periodic sides and no-slip walls (SIPG_BC_DIRICHLET,
 * g_u = 0); SIPG_BC_NEUMANN (outflow) sides are rejected.  Until `order`
 * levels are known the order rises one step at a time. */
typedef struct sipg_ns sipg_ns; /* opaque, owned by the library */

typedef struct {
  int k;                    /* polynomial degree, 2..7 (the pressure data need k >= 2)   */
  double penalty;           /* penalty factor of the SIPG forms (>= 1 recommended)     */
  double nu;                /* kinematic viscosity, > 0                                 */
  double dt;                /* time step, > 0                                           */
  int order;                /* J = 1, 2 or 3                                            */
  double zeta;              /* div-div factor zeta_D >= 0 of Eq. (tauD); 0 = no penalty  */
  int pressure_precond;     /* SIPG_PC_JACOBI or SIPG_PC_GMG_F32                         */
  double rtol_pressure;     /* CG stopping tolerances (relative residual)              */
  double rtol_viscous;
  double rtol_projection;   /* per-cell tolerance of the local projection              */
  int maxit;                /* iteration bound of the pressure and viscous CG          */
  int maxit_projection;     /* iteration bound of each cell's projection CG            */
} sipg_ns_params;

typedef struct {
  int order;                /* BDF order used in this step                          */
  int pressure_iters, viscous_iters, projection_iters;
  double pressure_relres, viscous_relres;
} sipg_ns_stats;

/* Defaults: k = 3, penalty 1, nu = 1/180, dt = 1e-3, order 3, zeta 1, Jacobi,
 * tolerances 1e-10 (pressure, viscous) and 1e-10 (projection), maxit 10000,
 * projection maxit 500. */
int sipg_ns_default_params(sipg_ns_params* prm);

/* Create a stepper on the current device for the velocity boundaries of desc
 * (the pressure mesh swaps no-slip walls for Neumann sides).  Allocates
 * about 18 velocity-sized vectors.  Errors: EINVAL, ENOMEM, ECUDA. */
int sipg_ns_create(const sipg_mesh_desc* desc, const sipg_ns_params* prm, sipg_ns** out);
int sipg_ns_destroy(sipg_ns* ns);

/* The stepper's meshes (owned by the stepper): which = 0 velocity (walls
 * Dirichlet), 1 pressure (walls Neumann).  Same geometry and node order. */
int sipg_ns_mesh(sipg_ns* ns, int which, sipg_mesh** out);

/* Set time level n - level (level 0 = the current velocity; level 0 resets the
 * history to one level, level i > 0 then adds older levels in order).
 * u: DEVICE, 3 * n_dofs doubles (components x, y, z), copied.  Computes the
 * level's convective term and wall data.  Synchronous. */
int sipg_ns_set_velocity(sipg_ns* ns, int level, const double* u, void* stream);

/* Advance one step with the body force f (HOST, 3 doubles, or NULL = 0) at
 * t^(n+1).  Synchronous (the solves read convergence data).  stats (HOST) may
 * be NULL.  Returns SIPG_MAXITER if a solve stopped at its bound (the step is
 * completed with the last iterates), the solvers' statuses otherwise.  After
 * any other error the stepper forgets its history (a slot may hold part of
 * the new level): set the velocity levels again before the next step. */
int sipg_ns_step(sipg_ns* ns, const double* f, void* stream, sipg_ns_stats* stats);

/* Copy the current velocity (3 * n_dofs) or pressure (n_dofs) to DEVICE
 * memory of the caller.  The pressure is determined up to an additive
 * constant (Neumann walls and periodic sides): the zero-mean CG fixes its
 * residual, not its mean. */
int sipg_ns_velocity(const sipg_ns* ns, double* u, void* stream);
int sipg_ns_pressure(const sipg_ns* ns, double* p, void* stream);

/* The wall data (div F^c(u) + nu curl omega) . n of the current velocity at
 * the (k+1)^2 Gauss points of every wall face (DEVICE, *count doubles; faces
 * ordered by cell, then direction, then low/high side; points with the first
 * tangential direction fastest).  h may be NULL to query *count (HOST). */
int sipg_ns_wall_data(const sipg_ns* ns, double* h, long long* count, void* stream);

/* Size in bytes of the static workspace of sipg_cg_solve_noalloc (host output). */
int sipg_cg_noalloc_capacity(long long* bytes);

/* Adjoint gradient for a per-cell viscosity (not in the paper; the operator is
 * the one of Sec. 3.2 (iii) in Laplace form): grad[e] = - lambda^T (dA/dnu_e) u
 * for A(nu) = mass_coef M + L(nu), with lambda the solution of the adjoint
 * system A lambda = dJ/du.  nu_cell, u, lambda: DEVICE (ncell, n_dofs, n_dofs
 * doubles, one component); grad: DEVICE, ncell doubles.  On a face where the
 * two viscosities are equal the penalty derivative is split half and half. */
int sipg_adjoint_grad_nu(const sipg_mesh* mesh, const double* nu_cell, const double* u, const double* lambda,
                         double* grad, void* stream);

/* Choose the cells-per-block of the operator kernels for this mesh and
 * precision (0 = FP64, 1 = FP32, also choosing the FP32 thread mapping) by
 * timing the candidates with CUDA events.  If cache_path is not NULL the
 * choice is read from / stored in that JSON file, an object with one entry
 * "k=<k> prec=<precision> map=<map> n=<nx>x<ny>x<nz>[ arith=native|df]":
 * {"cpb": <cells per block>, "mapping": <sipg_threads>} per configuration
 * (the file is rewritten whole on every store; a file of another shape counts
 * as empty).  precision 2 tunes the convective kernel; the FP64 keys include
 * the mesh's current FP64 arithmetic. */
int sipg_autotune(sipg_mesh* mesh, int precision, const char* cache_path);

/* Arithmetic of the FP64 operator entry points (sipg_apply_laplace_f64,
 * sipg_apply_helmholtz_f64 and the operator inside sipg_cg_solve).  SIPG_F64_NATIVE (default) computes in
 * FP64.  SIPG_F64_DOUBLE_FLOAT keeps the FP64 data in memory but evaluates the
 * sum-factorised operator in double-float arithmetic (pairs of FP32 with exact
 * product errors and TwoSum, about 2^-46 relative per operation) on the FP32
 * pipes, which issue 64 times the FP64 rate on GB300; results stay within the
 * FP64 parity tolerance (1e-12 of ||A|| ||x||).  The same choice applies to
 * sipg_apply_inverse_mass_f64 (and the inverse-mass preconditioner), to the
 * per-cell-viscosity Helmholtz operator, to sipg_apply_mass_f64, to the
 * general-map operator, the convective term, the viscous coupling and the
 * local div-div projection; the diagonal and the adjoint-gradient kernels
 * always use FP64.
 *
 * Range: every double-float call first reduces the largest exponent of the
 * finite entries of its FP64 input (one extra pass over the input, or, inside
 * CG, in the search-direction update) and evaluates input * 2^-s with
 * max |input| 2^-s in [1/2, 1), scaling the results back by the exact power
 * of two.  FP64 data anywhere in the FP64 range (subnormals included) keep
 * their 48 bits; entries below 2^-103 of the call's largest entry count as 0,
 * far below the tolerance.  NaN and +-inf in the input give NaN / +-inf in the
 * outputs they reach (as in FP64), so a CG solve from a non-finite x0 returns
 * SIPG_NONFINITE.  Scalar coefficients (mass_coef, nu, mass_coef / nu) must
 * be 0 or lie in [2^-100, 2^100] in magnitude, else the call returns
 * SIPG_EINVAL (use SIPG_F64_NATIVE); per-cell coefficient arrays (nu_cell, tau)
 * are converted unscaled: their nonzero entries must lie in [2^-100, 2^126].
 * The scale lives in a 16-byte word of the mesh (allocated by
 * sipg_create_mesh), so double-float calls on one mesh must be ordered on the
 * GPU (one stream, or streams joined by events). */
int sipg_set_f64_arithmetic(sipg_mesh* mesh, int mode);
int sipg_get_f64_arithmetic(const sipg_mesh* mesh, int* mode);

/* Thread mapping of the FP32 operator with a uniform viscosity:
 * SIPG_THREADS_LINE (default: p^2 threads per cell, one line each) or
 * SIPG_THREADS_PLANE (p threads per cell, one plane of p lines each, so that
 * every 1D matrix is loaded once per p lines; slower on GB300 at k = 4, 5 in
 * our measurements, kept for the autotuner).  Same results.  Resets the FP32 cells
 * per block to the mapping's default; sipg_autotune(precision 1) searches both
 * mappings. */
typedef enum { SIPG_THREADS_LINE = 0, SIPG_THREADS_PLANE = 1 } sipg_threads;
int sipg_set_f32_mapping(sipg_mesh* mesh, int mapping);

/* Cells per block currently used for a precision (host output).  precision
 * 2 addresses the kernel of sipg_apply_convective_f64 (cells of one thread
 * block; 0 < cpb <= the count whose shared memory fits 200 KB). */
int sipg_get_cells_per_block(const sipg_mesh* mesh, int precision, int* cpb);
int sipg_set_cells_per_block(sipg_mesh* mesh, int precision, int cpb);

/* Timing of the operator kernels: when enabled, CUDA events bracket every
 * operator-apply launch issued by the library on the caller's stream, and
 * sipg_profile_read returns the summed event time (ms), the number of timed
 * applies and the number of kernels the library launched since the last reset
 * (all kernels, timed or not).  Enabling adds an event record around each
 * apply; it is off by default.  Graph replays are not bracketed. */
int sipg_profile_enable(sipg_mesh* mesh, int on);
int sipg_profile_read(sipg_mesh* mesh, int reset, double* apply_ms, long long* applies, long long* launches);

/* Thread-local message describing the last error ("" if none). */
const char* sipg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SIPG_H */
