/*
 * pmgfr.h -- C interface of the GB300 implicit P-multigrid flux
 * reconstruction library (libpmgfr.so).
 *
 * The library solves the compressible Euler and Navier-Stokes equations (2D
 * quadrilaterals; hexahedra with pmg_config.dim = 3) with
 * Weiss-Smith/Turkel local preconditioning, discretised by FR/CPR
 * (Gauss-Legendre solution points, DG/Radau correction functions) and advanced
 * by ESDIRK2, 3 or 4 with dual time stepping.  Each implicit stage is solved by
 * pseudo-transient continuation whose pseudo-iteration is one FAS V-cycle over
 * polynomial levels with an element-Jacobi smoother (Wang & Yu, arXiv
 * 1908.03972, Sections 2-3), or, chosen with pmg_set_stage_solver, by
 * Newton-Krylov with that V-cycle as the preconditioner.
 *
 * Conventions shared by every call
 *  - Working variables are primitive q_p = (p, u, v, T) with R = 1
 *    ((p, u, v, w, T) on hexahedra).
 *  - A state array of level l is FP64, variable-major ("SoA"):
 *      q[(v * E + e) * N + pt],  v in 0..3, N = (P_l + 1)^2,
 *    and solution point (i, j) of an element has pt = j * (P_l + 1) + i with
 *    i along the first reference direction xi (hexahedra: v in 0..4,
 *    N = (P_l + 1)^3, pt = (k * (P_l + 1) + j) * (P_l + 1) + i).
 *  - Pointers flagged by on_device = 1 are caller-owned device buffers on the
 *    context's device; on_device = 0 means caller-owned host memory.  The
 *    library copies what it needs and never keeps caller pointers.
 *  - Every call is ordered on the CUDA stream given to pmg_create.  Calls
 *    that return host data synchronise that stream.
 *  - Every call returns a pmg_status; PMG_OK is 0 and errors are negative.
 *    pmg_last_error() gives a message for the calling thread's last error.
 *    No C++ exception crosses this interface.  There is no CPU fallback: if
 *    the GPU path cannot run, the call fails with PMG_ECUDA.
 */
#ifndef PMGFR_H
#define PMGFR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pmg_ctx pmg_ctx; /* opaque, owned by the library */

typedef enum {
  PMG_OK = 0,
  PMG_EINVAL = -1,     /* bad argument, size or call order */
  PMG_ENOMEM = -2,     /* device allocation failed */
  PMG_ECUDA = -3,      /* CUDA runtime error (message in pmg_last_error) */
  PMG_ESINGULAR = -4,  /* an element block is singular to working precision */
  PMG_ENONFINITE = -5, /* non-finite residual norm */
  PMG_ENOTCONV = -6,   /* stage did not reach the tolerance in max_pseudo */
  PMG_ETIMEOUT = -7,   /* a kernel's bounded wait for a bulk shared-memory
                          copy gave up (the kernel finished from global memory,
                          so the results are still those of the method) */
  PMG_ESTATE = -8      /* call needs data that was not set (mesh, stage) */
} pmg_status;

/* Precision of the element-Jacobi smoother's blocks (Section 2.4, eq.
 * smoothing_element_jacobi: the smoother needs only an approximate inverse).
 * Every sweep applies the inverse to the level-system residual F - S formed
 * in the residual arithmetic (flux_prec) and adds the result to the binary64
 * state, so each sweep is one step of a defect correction whose fixed point
 * is that of F alone: the block precision changes the contraction, not the
 * converged state. */
typedef enum {
  PMG_PREC_FP64 = 0, /* blocks factored and applied in FP64 */
  PMG_PREC_FP32 = 1, /* blocks equilibrated, factored and applied in FP32 */
  PMG_PREC_BF16R = 2 /* blocks equilibrated and factored in FP32, the inverse
                        stored in BF16 (half the bytes every sweep reads) and
                        applied with FP32 accumulation */
} pmg_prec;

/* Arithmetic of the residual.  Double-word (float-float) arithmetic runs the
 * common Roe flux (eq. invis_com) on the FP32 pipes at ~2^-46 relative
 * rounding, with the face traces, the jumps it takes and the central pressure
 * term in binary64; with gauge storage (p_gauge != 0) and mu = 0 the
 * residual-and-update of the element-Jacobi sweeps (the volume terms, the
 * level-system epilogue) is double-word too.  The sweeps are the smoother
 * and the coarse levels only shape the FAS corrections of Section 3; the
 * finest level's residual defines the converged solution: the stopping
 * norm, the defect restricted to the coarse levels and pmg_residual. */
typedef enum {
  PMG_FLUX_FP64 = 0,      /* binary64 everywhere */
  PMG_FLUX_DW_SMOOTH = 1, /* double-word in every sweep and in the coarse
                             levels' residuals, binary64 in the finest
                             level's residual: the converged state solves
                             the binary64 residual equations */
  PMG_FLUX_DW = 2         /* double-word in every residual */
} pmg_flux_prec;

/* Solver configuration (Sections 2.2-3, 4.1).
 *  P[l], n_smooth[l]: the hierarchy P{P0-P1-...} and the smoothing counts
 *  I{n0-n1-...}; pre- and post-smoothing use the same count, the coarsest
 *  level smooths once (Section 3).  0 <= P <= 5, 1 <= n_levels <= 8.
 *  cutoff = 1: eps = min(1, max(kappa Ma_inf, Ma)) (eq. eps_nonmove);
 *  cutoff = 0: eps = min(1, Ma) (Section 4.1).
 *  dtau_init, dtau_max, refresh_every: pseudo time step control (eq. ser
 *  with dtau set directly; smoother rebuilt at the first pseudo-iteration of
 *  a stage, then every refresh_every iterations until one rebuild used
 *  dtau_max).  tol: relative drop of ||F|| that ends a stage. */
typedef struct {
  int n_levels;
  int P[8];
  int n_smooth[8];
  double gamma, Ma_inf, kappa;
  int cutoff;
  double dtau_init, dtau_max, tol;
  int refresh_every, max_pseudo;
  int block_prec; /* pmg_prec */
  int use_graph;  /* 1: replay each V-cycle as a captured CUDA graph */
  double p_gauge; /* reference pressure kept out of device storage: the
                     library stores p - p_gauge (0: p itself) and uses it in
                     the momentum flux, where the constant part only adds
                     p_gauge times the discrete metric identity.  At low Mach
                     a value near the free-stream pressure keeps the pressure
                     resolution at the level of its variations.  Curved
                     (geom_order > 1) meshes need P >= geom_order on the
                     finest level (pmg_upload_mesh returns PMG_EINVAL
                     otherwise).  A coarser level with P < geom_order gets
                     a constant p_gauge times its metric-identity residual
                     back in the residual calls; the V-cycle's FAS equations
                     do not depend on it.  Every call still takes and
                     returns absolute p. */
  double mu;      /* constant dynamic viscosity (Section 2.1); 0: Euler.
                     mu > 0 adds the viscous fluxes with the common
                     solution of eq. com_q and the BR2 common gradient of
                     eq. com_grad_q (penalty eta_f = 4, the number of faces
                     of a quadrilateral) to the residual and to the element
                     blocks.  The fused coarse sweep is not used then. */
  double Pr;      /* Prandtl number of the heat flux K_j = -(mu Cp / Pr)
                     dT/dx_j (0.72 in the paper); read when mu > 0 */
  double res_scale[4]; /* reference scale of each equation (mass, x and y
                     momentum, energy) in ||F||, the norm of eq. ser and of
                     the stopping test: ||F||^2 = sum_v sum_pts
                     (F_v / res_scale[v])^2 over the finest level.  The paper
                     leaves the weighting open; a value <= 0 counts as 1.
                     The free-stream convective flux scales (rho U, rho U^2,
                     rho U^2, rho U H) make the equations commensurate at low
                     Mach, where the unweighted norm is the energy residual,
                     H ~ 1/Ma^2 times any mass imbalance, and stages that
                     start near their solution stall. */
  double q_inf[4]; /* free-stream primitive state (p absolute, u, v, T) that
                     far-field boundary faces see as their outer state */
  int cfl_mode;   /* 0: dtau_init/dtau_max as given.  1: the CFL form of
                     Section 2.4: at the start of every stage dtau_init =
                     cfl_init dtau_min and dtau_max = cfl_max dtau_min, with
                     dtau_min = min over elements of min((dx/(P+1))/(c+|v|),
                     (dx/(P+1))^2 rho/mu) on the finest level (dx: twice the
                     distance from the element's barycentre to its nearest
                     face; c + |v| the largest and rho the smallest value over
                     the element's points), so that SER acts on the CFL number.
                     The paper's wall-bounded cases use 1e2 and 1e5. */
  double cfl_init, cfl_max;
  int esdirk_order; /* ESDIRK scheme of pmg_esdirk_step (Section 2.4): 2
                     (three stages), 3 (four stages) or 4 (six stages);
                     0 means 3 */
  int refresh_always; /* 0: after the first pseudo-iteration of a stage the
                     smoother is rebuilt every refresh_every iterations until
                     one rebuild used dtau_max (the rule of Section 4.4);
                     1: every refresh_every iterations throughout the stage
                     (Section 4.1 states only the period) */
  int flux_prec;  /* pmg_flux_prec (the element blocks are always
                     differentiated in binary64) */
  double copy_wait_s; /* bound of each kernel's wait for its bulk
                     shared-memory copies, in seconds (0: one second).  A wait
                     that gives up sets a flag, the kernel reads the data from
                     global memory instead and waits (again bounded) for its
                     copies to land before it exits; the V-cycle calls then
                     return PMG_ETIMEOUT.  A negative value makes every such
                     wait give up at once: a diagnostic that runs the
                     global-memory path and the PMG_ETIMEOUT report. */
  int device_loop; /* 1 (with use_graph = 1): pmg_stage_solve and the stages
                     of pmg_esdirk_step run their pseudo-iterations as one
                     CUDA graph whose conditional WHILE node repeats {a
                     one-thread controller applying the SER, refresh and stop
                     rules; the V-cycle with or without smoother rebuild},
                     with one host synchronisation per stage instead of one
                     per V-cycle.  0: the host runs the loop.  Both follow the
                     same rules; dtau may differ in the last bits (device
                     pow). */
  int dim;        /* 2 (or 0): quadrilaterals, q_p = (p, u, v, T);
                     3: hexahedra, q_p = (p, u, v, w, T), Euler (mu = 0) or
                     Navier-Stokes (mu > 0, the same BR2 viscous terms),
                     binary64 residual throughout (flux_prec is not used),
                     0 <= P <= 3, slip-wall (mu = 0), no-slip-wall (eps
                     cut-off) and far-field boundary faces, dtau set
                     directly (cfl_mode = 0) */
  double res_scale3[5]; /* dim = 3: reference scale of each of the five
                     equations in ||F|| (res_scale is not used) */
  double q_inf3[5];     /* dim = 3: free stream (p absolute, u, v, w, T) of
                     far-field faces (q_inf is not used) */
} pmg_config;

/* Boundary types, in the second slot of a boundary face's neighbour entry
 * (whose element slot is -1).  The paper states no boundary treatment; a
 * ghost state enters the same common fluxes (Section 2.3):
 *  slip wall: (p, u - 2 u_n n, T), inviscid runs only (mu = 0);
 *  no-slip adiabatic wall: (p, -u, -v, T); its mean state has u = 0, so it
 *    needs the eps cut-off (cutoff = 1, kappa Ma_inf > 0);
 *  far field: q_inf.
 * For the viscous terms the ghost side mirrors the element (one-sided BR2
 * gradient), and walls carry no viscous energy flux. */
enum { PMG_BC_SLIP_WALL = 2, PMG_BC_NOSLIP_WALL = 3, PMG_BC_FARFIELD = 4 };

/* Mesh of quadrilaterals (dim = 2) or hexahedra (dim = 3) with Lagrange
 * geometry of order geom_order.
 *
 * Hexahedra (dim = 3):
 *  nodes: (n_elem, (geom_order+1)^3, 3) FP64, node (c*(Ng+1) + b)*(Ng+1) + a
 *         with a along xi, b along eta, c along zeta.
 *  nbr:   (n_elem, 6, 3) int32: for local face f = 2 d + s (d = 0 xi, 1 eta,
 *         2 zeta; s = 0 the -1 side, 1 the +1 side) the neighbour element, its
 *         local face and an orientation code o in 0..7: face point (a, b) (a
 *         along the first, b along the second of the face's two reference
 *         directions in increasing order) is the neighbour's point (a', b')
 *         with (s, t) = (o & 4) ? (b, a) : (a, b), a' = (o & 1) ? P - s : s,
 *         b' = (o & 2) ? P - t : t.  A boundary face has neighbour -1 and
 *         PMG_BC_SLIP_WALL or PMG_BC_FARFIELD in the face slot.
 *  Solution point (i, j, k) of a level has index (k*(P+1) + j)*(P+1) + i, and
 *  state arrays are variable-major over the five variables.
 *
 * Quadrilaterals (dim = 2), geom_order 1 or 2:
 *  nodes: (n_elem, (geom_order+1)^2, 2) FP64, element geometry nodes at
 *         equispaced reference positions, node b*(geom_order+1)+a, a along xi.
 *  nbr:   (n_elem, 4, 3) int32: for local faces 0 (eta=-1), 1 (xi=+1),
 *         2 (eta=+1), 3 (xi=-1): neighbour element, its local face, and 1 if
 *         the two faces number their points in opposite order.  A
 *         boundary face has neighbour element -1 and a PMG_BC_* type in the
 *         face slot (0 in the third); pmg_upload_mesh returns PMG_EINVAL for
 *         an unknown type, a slip wall with mu > 0, or a no-slip wall
 *         without the eps cut-off.
 * Both arrays are host memory, copied during the call. */
typedef struct {
  int n_elem;
  int geom_order;
  const double* nodes;
  const int* nbr;
} pmg_mesh;

typedef struct {
  int pseudo_iters[8]; /* V-cycles used by each implicit stage */
  double res_drop[8];  /* final ||F||/||F^0|| of each implicit stage */
  double ms_total;     /* wall time of the step on the stream, milliseconds */
  int n_vcycles;       /* total V-cycles of the step */
  int n_refresh;       /* smoother rebuilds of the step */
} pmg_step_stats;

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL
 * for the legacy default stream).  *out receives the context. */
pmg_status pmg_create(const pmg_config* cfg, void* stream, pmg_ctx** out);

/* Destroy a context and free its device memory.  NULL is ignored. */
void pmg_destroy(pmg_ctx* ctx);

/* Message of the calling thread's last failed call ("" if none). */
const char* pmg_last_error(void);

/* Upload the mesh; builds operator tables and metrics of every level (the
 * exact mapping evaluated at each level's own points, Section 2.3).  Must be
 * called once, before any state call. */
pmg_status pmg_upload_mesh(pmg_ctx* ctx, const pmg_mesh* mesh);

/* Physical coordinates of the solution points of a level into host memory
 * xy[(e * N + pt) * 2 + {0, 1}]. */
pmg_status pmg_point_coords(pmg_ctx* ctx, int level, double* xy);

/* Set / read the solution state of a level (SoA layout above). */
pmg_status pmg_set_state(pmg_ctx* ctx, int level, const double* q, int on_device);
pmg_status pmg_get_state(pmg_ctx* ctx, int level, double* q, int on_device);

/* R = -div f of eq. eqn:FR_diff at every solution point of the level for the
 * state q (FP64; Section 2.3, eqs. eqn:FR_diff, invis_com). */
pmg_status pmg_residual(pmg_ctx* ctx, int level, const double* q, double* R, int on_device);

/* Stage data of the finest level: src = (q_c^n + dt sum_j a_ij R^j)/(omega dt)
 * (SoA, level 0 size) and omega*dt of eq. ESDIRK_primitive. */
pmg_status pmg_set_stage(pmg_ctx* ctx, const double* src, double omega_dt, int on_device);

/* F_l(q) = -q_c(q)/(omega dt) + R_l(q) (+ src on level 0), eq. ESDIRK_primitive. */
pmg_status pmg_stage_residual(pmg_ctx* ctx, int level, const double* q, double* F, int on_device);

/* Assemble the element blocks D_e = Gamma/dtau + M/(omega dt) - dR_e/dq_e
 * (eqs. linearized_pseudo_transient_final, smoothing_element_jacobi) of a
 * level at its current state, exact own-element derivative with neighbours
 * frozen.  level = -1 assembles every level at its current state. */
pmg_status pmg_assemble_blocks(pmg_ctx* ctx, int level, double dtau);

/* Copy the assembled FP64 blocks of a level, row-major n x n per element,
 * n = 4 N, row/column index v * N + pt. */
pmg_status pmg_get_blocks(pmg_ctx* ctx, int level, double* D, int on_device);

/* Replace the assembled FP64 blocks of a level by caller data (same layout as
 * pmg_get_blocks), e.g. blocks formed or modified on the host.  The blocks
 * count as assembled and not factored.  Synchronises the stream. */
pmg_status pmg_set_blocks(pmg_ctx* ctx, int level, const double* D, int on_device);

/* Factor the assembled blocks of a level (or all, level = -1) in the
 * configured precision: power-of-two row/column equilibration, then
 * Gauss-Jordan elimination with partial pivoting to the explicit inverse,
 * one CTA per block, or a thread-block cluster of 2, 4 or 8 CTAs for blocks
 * one CTA's shared memory cannot hold (same arithmetic, same result).
 * Returns PMG_ESINGULAR, naming the element and level of the highest such
 * block (level-major order), if a pivot is not finite or not
 * above n eps of the working precision (the equilibrated rows have unit size
 * and a row that depends on others leaves a pivot of rounding size, so such a
 * block is singular to working precision); the library's V-cycle calls report
 * it the same way when they rebuild the smoother. */
pmg_status pmg_factor_blocks(pmg_ctx* ctx, int level);

/* x = D^-1 r per element with the factored blocks (SoA vectors). */
pmg_status pmg_apply_blocks(pmg_ctx* ctx, int level, const double* r, double* x, int on_device);

/* Restriction (L2 projection, Section 3) of a level-lf field to level lf+1,
 * and prolongation (interpolation) of a level-(lf+1) field to level lf. */
pmg_status pmg_restrict(pmg_ctx* ctx, int lf, const double* qf, double* qc, int on_device);
pmg_status pmg_prolong(pmg_ctx* ctx, int lf, const double* qc, double* qf, int on_device);

/* One FAS V-cycle (Section 3) on the finest-level state with the current
 * stage data and pseudo time step dtau; refresh = 1 rebuilds every level's
 * smoother on the way down.  *res_norm_out (may be NULL) receives ||F_0|| at
 * the start of the cycle (binary64 whatever flux_prec says).  The sweep
 * kernels wait for their shared-memory bulk copies with the bound copy_wait_s;
 * a wait that gives up is reported here (and by the calls below that run
 * V-cycles) as PMG_ETIMEOUT, after the kernels fell back to global loads. */
pmg_status pmg_vcycle(pmg_ctx* ctx, double dtau, int refresh, double* res_norm_out);

/* Pseudo-transient continuation of the current stage (Section 2.4) from the
 * finest-level state: V-cycles with SER growth of dtau until
 * ||F|| <= tol ||F^0||.  iters / drop (may be NULL) receive the V-cycle
 * count and the final relative drop.  PMG_ENOTCONV after max_pseudo. */
pmg_status pmg_stage_solve(pmg_ctx* ctx, int* iters, double* drop);

/* One physical step of size dt (eq. ESDIRK_ns) with the ESDIRK scheme that
 * esdirk_order selects (2, 3 or 4) from the finest-level state; the stage
 * initial guess is the previous stage's solution.  Inside the
 * step the finest-level system F = -q_c(q)/(omega dt) + R(q) + src is
 * evaluated as -(q_c(q) - q_c(q^n))/(omega dt) + R(q) + sum_j a_ij R^j/omega,
 * identical in exact arithmetic, with the energy difference formed from the
 * pressure difference so that rho E ~ 1/Ma^2 is never rounded. */
pmg_status pmg_esdirk_step(pmg_ctx* ctx, double dt, pmg_step_stats* stats);

/* Newton-Krylov stage solver (no part of the paper's method: its introduction
 * describes matrix-free Newton-Krylov solvers and its concluding section
 * names Newton-Krylov with the P-multigrid method as preconditioner as future
 * work).  Selected with pmg_set_stage_solver, it replaces the pseudo-transient
 * continuation in pmg_stage_solve and in every stage of pmg_esdirk_step:
 *
 *   Newton on F(q) = 0 (the stage system of pmg_set_stage / the ESDIRK
 *   stage): solve A delta = F(q), A = -dF/dq, to the relative tolerance eta
 *   by restarted FGMRES(krylov_dim) with right preconditioning, in the space
 *   where each equation is divided by its res_scale (the stage norm); then
 *   q += lam delta, lam starting at min(1, max_update / (the largest relative
 *   change of p or T)) and halved (at most max_backtrack times, the last
 *   trial kept) until ||F|| falls by the factor (1 - 1e-4 lam).  The stage ends
 *   when ||F|| <= tol ||F^0|| (PMG_OK), after max_newton steps (PMG_ENOTCONV)
 *   or on a non-finite norm (PMG_ENONFINITE).
 *   A z = -(F(q + h z) - F(q)) / h, h = delta0 / rms(z_v / state_scale_v),
 *   with F in binary64 whatever flux_prec says.
 *   Preconditioner PMG_NK_PC_BLOCK: z = D^-1 r with the finest level's
 *   element blocks at the Newton iterate and dtau_pc.  PMG_NK_PC_VCYCLE: one
 *   FAS V-cycle (the configured levels, smoothing counts and arithmetic) on
 *   the stage system with source src - F(q) + eps r from q, z = (q' - q)/eps,
 *   eps = pc_eps ||F(q)||; its blocks are rebuilt (all levels, dtau_pc) in the first
 *   application of every pc_refresh-th Newton step.
 *
 * With the Newton-Krylov solver pmg_step_stats.pseudo_iters counts Newton
 * steps and n_vcycles the preconditioner's V-cycles; pmg_stage_history holds
 * ||F|| after every Newton step (dtau entries 0 unless ptc_dtau > 0). */
typedef enum { PMG_STAGE_PTC = 0, PMG_STAGE_NK = 1 } pmg_stage_solver;
typedef enum { PMG_NK_PC_BLOCK = 0, PMG_NK_PC_VCYCLE = 1 } pmg_nk_precond;
typedef struct {
  int max_newton;          /* Newton steps per stage (<= 0: 30) */
  int krylov_dim;          /* FGMRES restart length m, 1..64 (<= 0: 20) */
  int max_krylov;          /* Krylov iterations per Newton step (<= 0: 2 m) */
  double eta;              /* relative tolerance of each linear solve (<= 0: 1e-2) */
  int precond;             /* pmg_nk_precond */
  double dtau_pc;          /* dtau in the preconditioner's blocks (<= 0: dtau_max) */
  int pc_refresh;          /* rebuild its blocks every pc_refresh Newton steps (<= 0: 1) */
  double delta0;           /* difference step of the Jacobian-vector product (<= 0: 1e-7) */
  double state_scale[5];   /* scale of each state variable for that step; an entry <= 0
                              takes the RMS of the variable over the stage's first
                              iterate (plus |p_gauge| for the pressure) */
  int max_backtrack;       /* step halvings of the line search (< 0: 6) */
  double max_update;       /* the line search starts from lam = min(1, max_update / r), r
                              the largest relative change |dp|/p, |dT|/T of any point
                              under the full correction (<= 0: 0.2): keeps p and T
                              positive far from the solution */
  double pc_eps;           /* V-cycle preconditioner: eps = pc_eps ||F(q)|| (<= 0: 0.1;
                              with 1 the V-cycle sees the whole Newton defect and
                              can leave its linear range) */
  double ptc_dtau;         /* > 0: pseudo-transient Newton (Kelley & Keyes): every
                              Newton step solves (Gamma(q)/dtau + A) delta = F, the
                              linearised backward-Euler step of the pseudo-time
                              system (eq. preconditioning), with dtau starting here
                              and following SER with exponent 1.5 and no upper
                              bound (dtau *= (||F_old|| / ||F_new||)^1.5); the
                              preconditioner takes min(dtau, dtau_pc), and the step
                              lam delta takes lam from the max_update limit alone
                              (no backtracking).  pmg_stage_history's dtau entries
                              hold each step's dtau.  <= 0 (default): Newton */
} pmg_nk_options;
typedef struct {
  long long newton;        /* Newton steps */
  long long krylov;        /* FGMRES iterations */
  long long vcycles;       /* preconditioner V-cycles */
  long long residuals;     /* binary64 stage-residual evaluations */
} pmg_nk_stats;

/* Choose the stage solver: PMG_STAGE_PTC (the default) or PMG_STAGE_NK with
 * options (opts may be NULL for the defaults; copied).  PMG_EINVAL for an
 * unknown solver or options out of range. */
pmg_status pmg_set_stage_solver(pmg_ctx* ctx, int solver, const pmg_nk_options* opts);

/* Counts of the Newton-Krylov work since the last reset (reset = 1 zeroes
 * them after the read).  Host memory. */
pmg_status pmg_nk_stats_read(pmg_ctx* ctx, pmg_nk_stats* out, int reset);

/* Residual norm ||F^m|| and pseudo time step of every pseudo-iteration of the
 * last pmg_stage_solve or pmg_esdirk_step (all stages, in order).  Up to
 * max_count entries are written to norms / dtau (either may be NULL);
 * *count receives the total number recorded.  Host memory. */
pmg_status pmg_stage_history(pmg_ctx* ctx, double* norms, double* dtau, int max_count, int* count);

/* Per-launch profiler.  While enabled, every kernel launch of the solver is
 * bracketed by CUDA events on the context's stream (V-cycles are then issued
 * launch by launch, not as a captured graph) and the event times are summed
 * per kernel class and level.  enable = 1 clears the sums. */
pmg_status pmg_profile(pmg_ctx* ctx, int enable);

/* Kernel classes of the profiler, in this order: face flux, volume residual,
 * block apply, block assembly, block factorisation, restriction, prolongation,
 * norm reduction, stage arithmetic, fused coarse-level sweep.  ms and counts
 * receive PMG_PROF_CLASSES x 8 entries (class-major, level 0..7): summed
 * milliseconds and launch counts. */
#define PMG_PROF_CLASSES 10
pmg_status pmg_profile_read(pmg_ctx* ctx, double* ms, long long* counts);

/* Autotuner of the coarse-level smoothing schedule (no counterpart in the
 * paper; the choice changes launch shapes, not the arithmetic).  For every
 * level that the double-word coarse-level kernels can serve (2D, a coarse
 * level with P <= 1, gauge storage, mu = 0, no boundary faces, flux_prec not
 * PMG_FLUX_FP64) it times the level's n_smooth sweeps, once untimed and
 * `reps` times between CUDA events on the context's stream, under each
 * candidate: the split face and volume launches (P = 1 only), one fused
 * launch per sweep, and tiles of 16, 32 or 64 core elements with 2, 3 or 4
 * sweeps per launch (k_tile.cu; every choice gives the same states bit for
 * bit on the fused path).  It keeps the fastest per level, unless it beats
 * the schedule in place by 2% or less, which then stays.  With cache_path
 * (a host string, may be NULL) a choice found there for the same (P, elements,
 * n_smooth, block_prec, SM count) is applied without timing, and new choices
 * are appended.  Needs the stage data and a smoother built by a V-cycle with
 * refresh = 1; the levels' data is left as the sweeps leave it, so the next
 * V-cycle recomputes what it uses.  report (may be NULL) receives the choice
 * and the timings per level. */
typedef struct {
  int n_levels;
  int fused[8];        /* 1: one launch per sweep or tiles; 0: split launches */
  int tile_core[8];    /* core elements per tile (0: no tiles) */
  int tile_depth[8];   /* sweeps per launch (0: no tiles) */
  int candidates[8];   /* schedules timed (0: level not tunable) */
  double us_per_sweep[8];        /* time per sweep of the choice, microseconds */
  double us_per_sweep_before[8]; /* time per sweep of the schedule in place before the call */
} pmg_tune_report;
pmg_status pmg_autotune(pmg_ctx* ctx, int reps, const char* cache_path, pmg_tune_report* report);

/* Allocation-free variant of pmg_residual, for callers that must not
 * allocate device memory once they are running: for example an application
 * that has handed all spare device memory to its own pool, or that runs under
 * a device-memory budget fixed at start-up.  (The paper has no counterpart;
 * this is an interface addition of this library.)
 *
 * Computes R = -div f exactly as pmg_residual does, for a state q and an
 * output R that are both caller-owned DEVICE buffers of the level's SoA size
 * on the context's device, which must be the current device.  The call makes
 * no cudaMalloc, cudaFree or other allocating call, on the device or the
 * host.  Its scratch is a copy of q and the common face fluxes, 4 E N +
 * 16 E (P+1) doubles, plus with mu > 0 the broken gradients and face jumps of
 * the viscous terms, 6 E N + 12 E (P+1) more (hexahedra: 5 E N + 30 E NF,
 * and 12 E N + 24 E NF, NF = (P+1)^2).  It lives in one static device
 * array of 2^21 doubles (16 MiB) that every GPU loading this library holds
 * until the process exits; a level that needs more returns PMG_EINVAL with
 * the sizes in the message.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for that device and keeps it for the life of the
 * process, so make the first call before any stream capture, and do not
 * reset the device (cudaDeviceReset) between calls.  All calls share the
 * array and each overwrites all of the scratch it reads, so nothing carries
 * over between calls; but calls whose GPU work overlaps (other streams, other
 * contexts, other host threads) race on it.  The call synchronises the
 * context's stream before returning. */
pmg_status pmg_residual_static(pmg_ctx* ctx, int level, const double* q, double* R);

/* Checkpoint and restore of the finest-level state (no counterpart in the
 * paper).  pmg_checkpoint writes a binary file at `path` (a host string): a
 * header (magic "PMGFRCK1", version, element count, geometry order, P of
 * every level, hashes of the mesh and of the discretisation settings gamma,
 * Ma_inf, kappa, cutoff, p_gauge, mu, Pr, res_scale and the P hierarchy) and
 * the state as stored on the device (variable-major FP64, pressure relative
 * to p_gauge).  Everything else a physical step uses (stage data, blocks,
 * coarse states) is rebuilt by the step, so a restored context repeats the
 * next pmg_esdirk_step bit for bit on the same GPU.  pmg_restore checks the
 * header against the context and returns PMG_EINVAL for another mesh, P
 * hierarchy or setting, a truncated or foreign file; PMG_ESTATE without a
 * mesh.  Both synchronise the context's stream. */
/* dtau_min of the CFL form (see cfl_mode) for the current finest-level state,
 * into *out (host).  Synchronises the context's stream.  PMG_ESTATE without a
 * mesh. */
pmg_status pmg_dtau_min(pmg_ctx* ctx, double* out);

pmg_status pmg_checkpoint(pmg_ctx* ctx, const char* path);
pmg_status pmg_restore(pmg_ctx* ctx, const char* path);

#ifdef __cplusplus
}
#endif
#endif /* PMGFR_H */
