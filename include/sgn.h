/*
 * sgn.h -- C ABI of the GB300 Sparse Gauss-Newton (SGN) library (libsgn.so).
 *
 * Problem (Zehnder, Coros, Thomaszewski, "SGN: Sparse Gauss-Newton for
 * Accelerated Sensitivity Analysis", ACM TOG 2021; Sec. 3, Eq. optProb):
 *     min_{x,p} f(x, p)   s.t.   c(x, p) = 0,   n_c = n_x,  dc/dx full rank,
 * where x are the free node positions of an elastic body, p one log-Young's
 * modulus per element (E_e = E0 exp(p_e)), c = dPi/dx the equilibrium
 * residual of the compressible neo-Hookean potential
 *     Pi = sum_e vol_e Psi(F_e) - f_ext . x,
 *     Psi(F) = mu/2 (tr F^T F - d) - mu ln J + lambda/2 (ln J)^2,
 * and f the nonlinear least-squares objective (Eq. leastSquaresObjective)
 *     f = 1/2 sum_t w_t (x_t - target_t)^2 + alpha/2 ||p||^2.
 *
 * The SGN step (Sec. 4, Eq. sparseSystemGN) solves the sparse saddle-point
 * system
 *     [ A   B^T  K^T  ] [dx]        with A = d2f/dx2 = diag(w) on tracked DOFs,
 *     [ B   C    cp^T ] [dp] = rhs       B = d2f/dp dx = 0, C = alpha I,
 *     [ K   cp   0    ] [dl]             K = dc/dx, cp = dc/dp,
 * whose dp equals the dense Gauss-Newton step H_GN dp = -df/dp^T
 * (Eq. newtonStep; Theorem 1 of Appendix A).
 *
 * Conventions for every call below
 *  - Arrays named *_h are host memory, *_d device memory on the device that
 *    was current at sgn_bind.  Device pointers are borrowed: the caller owns
 *    them and keeps them alive until the stream has passed the call.
 *  - Node-major layouts: positions, forces, dx and dlambda are [n_nodes][dim]
 *    doubles (fixed nodes: their prescribed position / zero step); p and dp
 *    are [n_elem] doubles.
 *  - Device work is enqueued on the stream given to sgn_bind / sgn_set_stream
 *    and is asynchronous unless a report is requested (reports synchronise).
 *  - Every call returns an sgn_status; a device-detected error (an inverted
 *    element, a non-finite value) is returned by the next call that
 *    synchronises.  sgn_strerror() gives a message.  No call aborts.
 *  - No call allocates device memory: the caller provides one device buffer
 *    of sgn_device_bytes() bytes at sgn_bind and the library carves its
 *    matrices, factors and workspaces out of it.
 */
#ifndef SGN_H
#define SGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SGN_OK = 0,
  SGN_EINVAL = 1,     /* bad argument (sizes, pointers, a partially fixed node ...) */
  SGN_ECUDA = 2,      /* a CUDA runtime call failed */
  SGN_ENOMEM = 3,     /* the bound device buffer is too small / host allocation failed */
  SGN_EINVERTED = 4,  /* an element has det F <= 0 at the given positions */
  SGN_ENEWTON = 5,    /* equilibrium Newton did not converge */
  SGN_EPIVOT = 6,     /* a pivot had to be perturbed and refinement did not recover */
  SGN_EREFINE = 7,    /* iterative refinement did not reach its tolerance */
  SGN_ESTATE = 8,     /* call out of order (e.g. solve before factor) */
  SGN_ENONFINITE = 9, /* a NaN or Inf reached a reduction */
  SGN_ETIMEOUT = 10   /* a bounded device-side wait expired (reported, never hangs) */
} sgn_status;

/* Precisions of the numeric factorization (sgn_factor). */
typedef enum {
  SGN_FP64 = 0,       /* fronts, pivots and Schur updates in FP64 (DFMA) */
  SGN_MIXED = 1       /* fronts in FP32; Schur updates on the tcgen05 tensor cores
                         as 3xTF32 products with FP32 accumulation; FP64 pivot
                         decisions, FP64 residuals and FP64 refinement */
} sgn_precision;

/* Right-hand side of Eq. sparseSystemGN (sgn_solve). */
typedef enum {
  SGN_RHS_KKT = 0,    /* [-f_x; -f_p; 0]: Newton-KKT form (Appendix A, Thm 2) */
  SGN_RHS_PAPER = 1   /* [0; -g; 0] with g = df/dp given by the caller (Eq. sparseSystemGN) */
} sgn_rhs_mode;

/* Device storage classes requested at sgn_device_bytes / sgn_bind. */
enum {
  SGN_STORE_FP64 = 1,   /* FP64 saddle-point fronts (SGN_FP64 factor) */
  SGN_STORE_MIXED = 2,  /* FP32 saddle-point fronts (SGN_MIXED factor) */
  SGN_STORE_KFACT = 4,  /* FP64 fronts of K alone (sgn_equilibrium, sgn_gradient) */
  SGN_STORE_KFACT_MIXED = 8  /* FP32 fronts of K alone (sgn_equilibrium with precision SGN_MIXED) */
};

typedef struct sgn_ctx *sgn_t;

/* Mesh and material (host arrays, copied by sgn_setup). */
typedef struct {
  int32_t dim;               /* 2 (plane-strain triangles) or 3 (tetrahedra) */
  int32_t n_nodes;
  int32_t n_elem;
  const double *X_h;         /* [n_nodes][dim] rest positions */
  const int32_t *conn_h;     /* [n_elem][dim+1] node ids, positively oriented */
  const uint8_t *fixed_h;    /* [n_nodes]: 1 = Dirichlet-fixed node (all of its DOFs) */
  double E0;                 /* reference Young's modulus, E_e = E0 exp(p_e) */
  double nu;                 /* Poisson ratio */
} sgn_mesh;

/* Symbolic-phase options; zero-initialise for defaults. */
typedef struct {
  int32_t leaf_nodes;        /* nested dissection stops at <= leaf_nodes nodes (0: 16) */
  int32_t panel;             /* pivot panel width: 8, 16 or 32 (0: 32) */
  int32_t update_ctas;       /* CTAs of one tensor-core trailing-update launch, shared by the
                                level's active fronts; each CTA loops over its tiles
                                (0: one per SM) */
} sgn_setup_opts;

/* Least-squares objective (host arrays, copied by sgn_set_objective). */
typedef struct {
  int32_t n_track;
  const int64_t *track_dof_h; /* global DOF ids node*dim+comp; must be free DOFs */
  const double *target_h;     /* [n_track] */
  const double *weight_h;     /* [n_track] weights (negative ones make A indefinite: see
                                 sgn_factor_inertia) */
  double alpha;               /* Tikhonov weight, > 0 (C = alpha I) */
} sgn_objective;

typedef struct {
  int64_t n_nodes, n_free, n_elem;
  int64_t n_x, n_p, n_kkt;        /* n_kkt = 2 n_x + n_p */
  int64_t nnz_kkt;                /* nonzeros of the full symmetric saddle-point matrix without A
                                     (A adds one diagonal entry per tracked DOF) */
  int64_t n_supernodes, n_levels;
  int64_t max_front;              /* largest front order (reduced saddle-point system) */
  int64_t nnz_factor;             /* entries of L incl. diagonal (reduced saddle-point system) */
  double factor_flops;            /* flops of one numeric factorization (reduced system) */
  double kfactor_flops;           /* flops of one factorization of K alone */
  double setup_seconds;           /* wall time of the host symbolic phase */
} sgn_info;

typedef struct {
  int64_t n_pos, n_neg, n_zero;   /* inertia of the saddle-point matrix (incl. p pivots) */
  int64_t n_2x2;                  /* 2x2 Bunch-Kaufman pivots */
  int64_t n_perturbed;            /* pivots replaced by the static-pivot threshold */
  double seconds;                 /* device time of the factorization */
  int64_t tensor_core_updates;    /* trailing-update launches on the tcgen05 tensor cores */
} sgn_factor_report;

/* How sgn_solve reaches its tolerance with the factor as preconditioner.
 * Sec. 5 ("Solving the saddle point problem") falls back to BiCGSTAB
 * preconditioned by an LDL^T factor when the direct solve is not accurate
 * enough; here stationary FP64 refinement comes first and BiCGSTAB (FP64,
 * right-preconditioned by the factor, on the unstabilized matrix) takes over
 * when refinement stops contracting. */
typedef enum {
  SGN_SOLVE_AUTO = 0,      /* refinement; BiCGSTAB from its last iterate once a refinement step
                              shrinks the residual by less than half above 1e-11 ||b||, or
                              max_refine steps did not reach tol */
  SGN_SOLVE_REFINE = 1,    /* refinement only (SGN_EREFINE if it ends above 1e-8 ||b||) */
  SGN_SOLVE_BICGSTAB = 2   /* BiCGSTAB from the first preconditioned solve */
} sgn_solve_method;

typedef struct {
  int32_t max_refine;             /* FP64 refinement steps (default 0 -> 2 FP64 / 30 mixed) */
  double tol;                     /* stop at ||b - M z|| <= tol ||b|| (default 0 -> 1e-12, just above
                                     the FP64 round-off floor of the 40^3 system, ~1.4e-13) */
  int32_t method;                 /* sgn_solve_method (0: SGN_SOLVE_AUTO) */
  int32_t max_krylov;             /* BiCGSTAB iterations (default 0 -> 200) */
  int32_t regularized;            /* 1: solve the factored matrix itself, M + diag(eps_x, 0, -eps_lambda)
                                     (the step of an inertia-corrected factorization); 0: solve M */
} sgn_solve_opts;

typedef struct {
  int32_t refine_steps;           /* refinement steps taken */
  double residual;                /* final ||b - M z|| / ||b|| in FP64 */
  double seconds;
  double history[32];             /* ||b - M z|| / ||b|| after each of the first 32 solves */
  int32_t krylov_iters;           /* BiCGSTAB iterations taken (0: refinement sufficed) */
} sgn_solve_report;

/* Stabilization of the factored matrix (sgn_factor_ex): the factor is taken
 * of M + diag(eps_x 1, 0, -eps_lambda 1) (x, p, lambda blocks), as Sec. 5
 * does for the LDL^T that preconditions BiCGSTAB; residuals, refinement and
 * BiCGSTAB still use M itself, so the solution is that of M. */
typedef struct {
  double eps_x, eps_lambda;       /* >= 0; both 0: the factor of M (sgn_factor) */
} sgn_factor_opts;

typedef struct {
  int32_t max_iter;               /* default 0 -> 50 */
  double tol;                     /* ||c|| <= tol ||f_ext|| (default 0 -> 1e-10).  The iterate is the
                                     displacement x - X, so the round-off floor of ||c|| does not
                                     depend on where the body sits (measured: 1.3e-11 ||f_ext|| on a
                                     60 x 60 grid); for a tol below the floor, a residual a Newton
                                     step no longer halves also counts once below 1e-10 ||f_ext|| */
  int32_t precision;              /* SGN_FP64 (default): K factored in FP64 (SGN_STORE_KFACT);
                                     SGN_MIXED: K factored with FP32 fronts on the tensor cores
                                     (SGN_STORE_KFACT_MIXED) and every Newton direction refined
                                     in FP64 against the FP64 K until ||K dx + c|| <=
                                     min(0.1, ||c|| / ||f_ext||) ||c|| (at most 10 solves;
                                     the stagnation rule above only counts after a
                                     direction that met this bound) */
} sgn_newton_opts;

typedef struct {
  int32_t iters;
  int32_t converged;
  double residual;                /* final ||c|| / ||f_ext|| */
  double initial_residual;
  double seconds;
  int32_t solves;                 /* K solves (more than iters with FP32 fronts: refinement) */
  double history[32];             /* ||c|| / ||f_ext|| at iterate 0, 1, ... (first 32) */
  double step_length[32];         /* accepted line-search step t of iteration 1, 2, ... */
} sgn_newton_report;

/* ---- set-up -------------------------------------------------------------
 * sgn_setup: host-only symbolic phase (Sec. 4: the sparsity of Eq.
 * sparseSystemGN is fixed by the mesh): free-node numbering, nested
 * dissection of the node graph, elimination tree, supernodes, front index
 * maps, the fixed block pattern of K and its element slot map.  Copies the
 * mesh.  EINVAL on bad sizes/indices; ENOMEM on host allocation failure. */
sgn_status sgn_setup(const sgn_mesh *mesh, const sgn_setup_opts *opts, sgn_t *out);
sgn_status sgn_get_info(sgn_t h, sgn_info *out);
/* Bytes of device memory needed for the given SGN_STORE_* mask. */
sgn_status sgn_device_bytes(sgn_t h, int32_t stores, size_t *bytes);
/* Carves dev_buf (>= sgn_device_bytes, 256-byte aligned) and uploads the
 * static symbolic data on `stream` (a cudaStream_t, NULL = default stream).
 * The buffer stays owned by the caller and must outlive h's use. */
sgn_status sgn_bind(sgn_t h, void *dev_buf, size_t bytes, int32_t stores, void *stream);
sgn_status sgn_set_stream(sgn_t h, void *stream);
/* Objective of Eq. leastSquaresObjective (tracked coordinates + Tikhonov). */
sgn_status sgn_set_objective(sgn_t h, const sgn_objective *obj);
void sgn_destroy(sgn_t h);
const char *sgn_strerror(sgn_status s);
/* Detail of the last failed call on h (which CUDA call or check failed);
 * empty if none.  Owned by h, valid until the next call on h. */
const char *sgn_last_error(sgn_t h);
/* Self-test of the bounded device waits (the paper has no counterpart): runs
 * one substitution wait, on the first bound store, for a block value that
 * nothing publishes.  Returns SGN_ETIMEOUT after about a second when the
 * wait gave up and reported as designed (the status word is then cleared
 * and h stays usable); any other status means the bound or its report
 * failed.  ESTATE before sgn_bind. */
sgn_status sgn_selftest_wait_timeout(sgn_t h);

/* ---- hot path ------------------------------------------------------------
 * sgn_assemble: element kernels evaluate, at positions x_d and parameters
 * p_d, the blocks of Eq. sparseSystemGN: K = dc/dx (Sec. 3.1), cp = dc/dp
 * (Eq. dcdp; column e is element e's force since Psi is linear in E), and
 * the Schur complement cp C^{-1} cp^T of the p block; all are scattered into
 * the fixed pattern without atomics.  EINVERTED (at the next synchronising
 * call) if det F <= 0 anywhere. */
sgn_status sgn_assemble(sgn_t h, const double *x_d, const double *p_d);
/* sgn_factor: numeric LDL^T of the assembled saddle-point matrix.  The p
 * unknowns (C = alpha I diagonal) are eliminated first; the remaining
 * (x, lambda) system is factored supernode by supernode (multifrontal) with
 * Bunch-Kaufman 1x1/2x2 pivots restricted to each panel of the fully-summed
 * block.  report may be NULL (no synchronisation). */
sgn_status sgn_factor(sgn_t h, sgn_precision prec, sgn_factor_report *report);
/* sgn_factor_ex: sgn_factor of the stabilized matrix of sgn_factor_opts
 * (opts NULL: as sgn_factor).  EINVAL for a negative eps. */
sgn_status sgn_factor_ex(sgn_t h, sgn_precision prec, const sgn_factor_opts *opts, sgn_factor_report *report);
/* sgn_factor_inertia: the inertia test with diagonal regularization that
 * Sec. 5 ("Solving the saddle point problem") uses for its Newton-type
 * variants (after Han 1985): factor M, and while the inertia is not
 * (n_x + n_p, n_x, 0) -- i.e. the reduced Hessian is not positive definite
 * on the null space of the constraint Jacobian, as happens with an
 * indefinite A (negative tracking weights) -- refactor with delta added to
 * the x diagonal, delta = delta0, delta0 growth, delta0 growth^2, ...  The
 * chosen delta goes to *delta_h (0: M itself was fine); solve the
 * regularized system with sgn_solve_opts.regularized = 1.  EPIVOT if
 * max_tries factorizations did not reach the inertia. */
typedef struct {
  double delta0;                  /* first regularization (0: 1e-4 x the largest |tracked weight|) */
  double growth;                  /* factor between attempts (0: 10) */
  int32_t max_tries;              /* factorizations at most (0: 30) */
} sgn_inertia_opts;
sgn_status sgn_factor_inertia(sgn_t h, sgn_precision prec, const sgn_inertia_opts *opts, double *delta_h,
                              sgn_factor_report *report);
/* sgn_solve: (dx, dp, dl) of Eq. sparseSystemGN by forward, diagonal and
 * backward substitution with the factor, followed by FP64 iterative
 * refinement against the assembled matrix.  g_d = df/dp for SGN_RHS_PAPER
 * (ignored otherwise).  Any of dx_d / dl_d may be NULL.  Each level's
 * substitution is one launch whose CTAs wait, bounded, for the blocks they
 * depend on: ETIMEOUT if such a wait expired (the result is then invalid). */
sgn_status sgn_solve(sgn_t h, sgn_rhs_mode mode, const double *g_d, double *dx_d,
                     double *dp_d, double *dl_d, const sgn_solve_opts *opts,
                     sgn_solve_report *report);
/* sgn_step_host: sgn_assemble + sgn_factor + sgn_solve(SGN_RHS_KKT) on host
 * buffers, including the host->device copy of x_h, p_h and the
 * device->host copy of the step.  Synchronises. */
sgn_status sgn_step_host(sgn_t h, sgn_precision prec, const double *x_h, const double *p_h,
                         double *dx_h, double *dp_h, double *dl_h, sgn_solve_report *report);

/* sgn_step_graph: one SGN step -- sgn_assemble at (x_d, p_d), sgn_factor
 * (prec), the solve of Eq. sparseSystemGN with the Newton-KKT right-hand
 * side and exactly refine_steps FP64 refinement steps -- issued as a single
 * CUDA-graph launch on the handle's stream (the graph is captured on the
 * first call and replayed while the arguments stay the same).  Outputs as
 * in sgn_solve; dx_d / dl_d may be NULL.  If residual_h is non-NULL the call
 * synchronises and stores ||b - M z|| / ||b|| (FP64) there.  EINVAL for
 * refine_steps outside 0..64. */
sgn_status sgn_step_graph(sgn_t h, sgn_precision prec, int32_t refine_steps, const double *x_d, const double *p_d,
                          double *dx_d, double *dp_d, double *dl_d, double *residual_h);

/* sgn_export_kkt: copies the assembled saddle-point matrix of Eq.
 * sparseSystemGN (the last sgn_assemble) to host COO arrays, both triangles.
 * Unknown ids: x_{node,a} -> node*dim + a, p_e -> n_nodes*dim + e,
 * lambda_{node,a} -> n_nodes*dim + n_elem + node*dim + a (fixed nodes have no
 * entries).  Call with rows_h == NULL to get the entry count in *nnz; else
 * rows_h / cols_h / vals_h must hold *nnz entries.  Synchronises. */
sgn_status sgn_export_kkt(sgn_t h, int64_t *nnz, int64_t *rows_h, int64_t *cols_h, double *vals_h);

/* sgn_assemble_static: same result as sgn_assemble (x_d, p_d in; the
 * assembled blocks, right-hand-side terms and dc/dp of the handle out), but
 * the per-element state it passes from the element kernel to the slot
 * gather lives in a fixed 16 MB device array inside the library, not in the
 * caller's bound buffer.  The paper has no counterpart.  It serves callers
 * that must not allocate device memory, or have the runtime set any up, at
 * the point where they assemble, e.g. a solver loop inside a memory-capped
 * service whose allocator is frozen after start-up.  It does not shrink the
 * bound buffer: sgn_device_bytes still counts the element-state region,
 * which this entry point leaves unused.  The array belongs to the library's
 * device image: every GPU that loads libsgn.so holds it until the process
 * exits.  sgn_bind looks up its device address with the handle's device
 * current, so under CUDA's lazy module loading the array is set up inside
 * sgn_bind, never inside this call, which allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  Limit: (3 + (dim+1) dim) *
 * n_elem doubles <= 2^21, i.e. 139,810 tetrahedra or 233,016 triangles;
 * larger meshes get SGN_EINVAL (sgn_strerror says why).  All calls share the
 * array (it keeps the last call's contents; every entry is rewritten before
 * it is read, so nothing needs clearing): calls whose work overlaps on the
 * GPU, from any handle or stream, race on it. */
sgn_status sgn_assemble_static(sgn_t h, const double *x_d, const double *p_d);

/* ---- batched instances ----------------------------------------------------
 * The paper solves one design instance at a time (Sec. 5); these calls put n
 * independent instances behind one handle.  sgn_batch_setup joins the meshes
 * (node ids of instance i shifted by the nodes of instances 0..i-1, elements
 * likewise) and their objectives (tracked DOF ids shifted the same way) into
 * one disjoint system: its matrix is block diagonal by instance, so every
 * instance's (dx, dp, dlambda) is exactly its own SGN step (Eq.
 * sparseSystemGN), while the symbolic phase splits the node graph into its
 * connected components first (one subtree of one elimination forest per
 * instance) and every level's fronts of all instances share the launches.
 * Instances keep their own coordinates and may overlap in space.  All meshes
 * need the same dim, E0 and nu, all objectives the same alpha (EINVAL
 * otherwise); objectives may be NULL (then call sgn_set_objective with joined
 * DOF ids).  The objective given here is applied by sgn_bind.  Every other
 * call then works on the joined arrays: positions [sum n_nodes][dim], p
 * [sum n_elem], in instance order. */
sgn_status sgn_batch_setup(int32_t n, const sgn_mesh *meshes, const sgn_objective *objectives,
                           const sgn_setup_opts *opts, sgn_t *out);
/* Number of instances in *n (0: not a batched handle) and, if the arrays are
 * non-NULL, the n + 1 node and element offsets of the instances. */
sgn_status sgn_batch_info(sgn_t h, int32_t *n, int64_t *node_off_h, int64_t *elem_off_h);
enum {
  SGN_BATCH_EQUILIBRIUM = 0,  /* ||c_i|| / ||f_ext,i|| at the last sgn_equilibrium's iterate */
  SGN_BATCH_KKT = 1           /* ||b_i - M_i z_i|| / ||b_i|| of the last sgn_solve / sgn_step_graph */
};
/* Per-instance relative residuals (res_h: n doubles, FP64), synchronises.
 * ESTATE if no such call has run since sgn_bind. */
sgn_status sgn_batch_residuals(sgn_t h, int32_t kind, double *res_h);

/* ---- forward simulation and gradient -------------------------------------
 * sgn_equilibrium: Newton's method on Pi(x; p) with a backtracking line
 * search that keeps Pi monotone and rejects inverted elements (Sec. 5,
 * "Computing Equilibrium States"); K is factored with the same multifrontal
 * machinery (needs SGN_STORE_KFACT).  x_d: initial guess in, equilibrium
 * out.  fext_d: [n_nodes][dim] external forces.  Synchronises. */
sgn_status sgn_equilibrium(sgn_t h, const double *p_d, const double *fext_d, double *x_d,
                           const sgn_newton_opts *opts, sgn_newton_report *report);
/* sgn_gradient: total gradient df/dp = f_p + cp^T lambda_adj with the
 * adjoint lambda_adj = -K^{-T} f_x (Eq. totalGradient and the remark after
 * it: one linear solve, here with the K factor of sgn_factor_k).  Uses the
 * blocks and f_x, f_p of the last sgn_assemble; ESTATE if K is not factored
 * at that point.  g_d: [n_elem]. */
sgn_status sgn_gradient(sgn_t h, double *g_d);
/* sgn_factor_k: factor K alone at the assembled (x, p) (FP64). */
sgn_status sgn_factor_k(sgn_t h);

/* ---- SGN-initialised L-BFGS (Sec. 4, "Combination with L-BFGS") ----------
 * The Gauss-Newton inverse Hessian initialises L-BFGS: each search direction
 * is the two-loop recursion (Nocedal & Wright, Alg. 7.4) over the m most
 * recent pairs s = p_{k+1} - p_k, y = g_{k+1} - g_k with H_0^{-1} q applied
 * by one solve of Eq. sparseSystemGN (right-hand side [0; -q; 0]) with the
 * saddle-point factor of the current iterate.
 *
 * sgn_objective_value: f(x, p) of Eq. leastSquaresObjective at node
 * positions x_d and parameters p_d (synchronises). */
sgn_status sgn_objective_value(sgn_t h, const double *x_d, const double *p_d, double *f_h);
/* sgn_lbfgs_direction: d_d = -H_k g_d for the pairs s_d, y_d ([m][n_elem]
 * each, oldest first, y.s > 0) with H_0 = H_GN of the last sgn_assemble +
 * sgn_factor (ESTATE if that factor is not current).  m = 0 gives the SGN
 * step itself. */
sgn_status sgn_lbfgs_direction(sgn_t h, int32_t m, const double *s_d, const double *y_d, const double *g_d,
                               double *d_d);
typedef struct {
  int32_t m;                 /* pairs kept (0: plain SGN steps with the same line search) */
  int32_t max_iter;          /* outer iterations */
  double tol_g;              /* stop once ||df/dp|| <= tol_g (0: run max_iter) */
  int32_t precision;         /* saddle-point factor: SGN_FP64 or SGN_MIXED */
  int32_t eq_precision;      /* equilibrium Newton: SGN_FP64 or SGN_MIXED */
  double armijo;             /* sufficient-decrease constant (0: 1e-4) */
  int32_t max_halvings;      /* line-search trials (0: 30) */
} sgn_lbfgs_opts;
typedef struct {
  int32_t iters, converged, restarts;  /* restarts: steps that fell back to -g */
  int32_t trials, equilibrium_iters;   /* line-search trials, Newton iterations in all equilibria */
  double seconds;
  double f[64], gnorm[64];             /* f and ||df/dp|| at iterate 0, 1, ... */
  double step[64];                     /* accepted step length of iteration 1, 2, ... */
} sgn_lbfgs_report;
/* Device bytes sgn_optimize_lbfgs needs in work_d for m pairs. */
sgn_status sgn_lbfgs_work_bytes(sgn_t h, int32_t m, size_t *bytes);
/* sgn_optimize_lbfgs: L-BFGS iterations on p (device, in/out) for the
 * external load fext_d: every iterate's equilibrium x(p) by sgn_equilibrium
 * (x_d: initial guess in, the last iterate's equilibrium out), the adjoint
 * gradient (sgn_factor_k + sgn_gradient), the direction above, and a
 * backtracking line search on f(x(p), p) (Armijo; a trial whose Newton
 * fails counts as no decrease).  Needs SGN_STORE_KFACT and the saddle-point
 * store of opts->precision; work_d (caller-owned, sgn_lbfgs_work_bytes) holds
 * the pairs and vectors, so the call allocates nothing.  Synchronises. */
sgn_status sgn_optimize_lbfgs(sgn_t h, const double *fext_d, double *p_d, double *x_d, void *work_d,
                              size_t work_bytes, const sgn_lbfgs_opts *opts, sgn_lbfgs_report *rep);

/* ---- measurement support (no counterpart in the paper) ------------------
 * sgn_profile(h, mask) resets the per-kernel timers and enables CUDA-event
 * timing (on the context's stream) of every launch of the kernel kinds whose
 * bit is set in mask (mask = 0 disables).  sgn_profile_read synchronises and
 * fills out[k] for kind k < n: launches, summed device seconds, and summed
 * algorithmic flops (trailing and panel updates: 2 * rows * cols * inner
 * dimension of the lower-triangle update; 0 for the other kinds). */
enum {
  SGN_PROF_UPDATE = 0,          /* trailing Schur update of an outer block (dominant) */
  SGN_PROF_PANEL_UPDATE = 1,    /* left-looking update of a pivot panel */
  SGN_PROF_PIVOT = 2,           /* Bunch-Kaufman factorization of a panel's diagonal block */
  SGN_PROF_TRSM = 3,            /* L21 / W of a panel */
  SGN_PROF_FRONT_ASSEMBLY = 4,  /* front assembly (original entries + children) */
  SGN_PROF_ELEMENTS = 5,        /* element evaluation and block gather */
  SGN_PROF_SOLVE = 6,           /* forward / diagonal / backward substitution */
  SGN_PROF_VECTOR = 7,          /* right-hand sides, p elimination, residuals, reductions */
  SGN_PROF_KINDS = 8
};
typedef struct {
  int64_t launches;
  double seconds;
  double flops;
} sgn_kernel_profile;
sgn_status sgn_profile(sgn_t h, int32_t mask);
sgn_status sgn_profile_read(sgn_t h, sgn_kernel_profile *out, int32_t n);
/* Number of CUDA kernels this context has launched since sgn_bind. */
int64_t sgn_launch_count(sgn_t h);

#ifdef __cplusplus
}
#endif
#endif /* SGN_H */
