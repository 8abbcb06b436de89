/*
 * libsipg -- matrix-free SIPG operator and cph hybrid multigrid on one GB300.
 *
 * C ABI of the hot path of Fehn, Munch, Wall, Kronbichler, "Hybrid multigrid
 * methods for high-order discontinuous Galerkin discretizations"
 * (arXiv:1910.01900).  Every call is plain C: opaque context, plain pointers
 * and sizes, no C++ or framework types.
 *
 * Conventions that hold for every entry point
 * -------------------------------------------
 * - Return value: a sipg_status; SIPG_OK on success.  Nothing throws across
 *   this boundary.  sipg_last_error(ctx) returns a text for the last failure of
 *   that context (sipg_last_error(NULL): last failure of sipg_create).
 * - Vectors named *_dev are DEVICE pointers owned by the caller, on the device
 *   that was current when the context was created.  Vectors named *_host are
 *   host pointers owned by the caller.  The library never frees or keeps caller
 *   pointers after a call returns.
 * - DoF order of a DG vector (level L, the finest): cell-major with cells
 *   lexicographic (x fastest), then the (k+1)^3 nodes of the cell
 *   lexicographic (x fastest).  FE vectors (levels below L): the global grid
 *   of (m k'+1)^3 nodes, lexicographic, x fastest.
 * - precision argument: 0 = double (FP64), 1 = float (FP32).  A void* vector
 *   holds elements of that type.
 * - All work is ordered on the context's stream (sipg_params.stream; NULL =
 *   the legacy default stream).  Calls that return numbers to the host
 *   (solve info, norms) synchronize that stream; all others are asynchronous.
 * - The library owns every internal buffer (allocated in sipg_create, freed in
 *   sipg_destroy).  Calls on one context must not overlap in time from
 *   different host threads.
 */
#ifndef SIPG_H
#define SIPG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sipg_ctx sipg_ctx;

typedef enum {
  SIPG_OK = 0,
  SIPG_EINVAL = 1,      /* bad argument: size, degree, pointer, precision    */
  SIPG_ECUDA = 2,       /* a CUDA runtime call failed                         */
  SIPG_ENOMEM = 3,      /* device or host allocation failed                   */
  SIPG_ENOTCONV = 4,    /* solver hit maxit before reaching the tolerance     */
  SIPG_EBREAKDOWN = 5,  /* p^T A p <= 0 or a non-finite scalar in the solver  */
  SIPG_ETIMEOUT = 6,    /* a bounded device-side wait ran out                 */
  SIPG_ENAN = 7         /* non-finite input (right-hand side norm)           */
} sipg_status;

/* Structured hexahedral box mesh (Section 2: hexahedral cells, mapping x(xi)
 * from the reference cell [0,1]^3; Section 5.3: deformed cube with degree-3
 * element mappings).  m[i] cells in direction i over [lo_i, hi_i].
 * deform = 0: affine (Cartesian) cells.  deform = 1: every cell is the
 * tensor Lagrange interpolant of degree mapping_degree (must be 3) on its GL
 * points of the map x_i <- x_i + amp * prod_j sin(pi (x_j-lo_j)/(hi_j-lo_j)).
 * bc[s] for the box sides s = -x,+x,-y,+y,-z,+z: 0 = Dirichlet, 1 = Neumann
 * (Eq. BoundaryConditions; only the homogeneous operator is applied). */
typedef struct {
  int m[3];
  double lo[3], hi[3];
  int deform;
  double amp;
  int mapping_degree;
  int bc[6];
} sipg_mesh;

/* Unstructured hexahedral mesh (Section 2; Section 5.3: the paper's nozzle
 * and lung meshes are unstructured hexahedra with Dirichlet and Neumann
 * boundary parts).  Host arrays, read during sipg_create_unstructured only:
 * vertices [nverts][3]; cells [ncells][8] vertex ids, local vertex i + 2 j +
 * 4 k at the reference corner (i, j, k) of [0,1]^3, the cell map being the
 * trilinear interpolant of the 8 vertices; face_bc [ncells][6] for the local
 * face f = 2 d + s (the face xi_d = s): 0 Dirichlet, 1 Neumann on boundary
 * faces, ignored on interior faces (NULL: every boundary face Dirichlet).
 * Two cells are neighbours through a face whose four vertex ids both hold;
 * any relative orientation of the two cells is allowed.  deform = 1 applies
 * x_i += amp * prod_j sin(pi (x_j-lo_j)/(hi_j-lo_j)) to the trilinear image,
 * interpolated at degree 3 on the cell's GL points (as sipg_mesh). */
typedef struct {
  int nverts;
  const double *vertices;
  int ncells;
  const int *cells;
  const int *face_bc;
  int deform;
  double amp;
  double lo[3], hi[3];
} sipg_hex_mesh;

/* Method parameters (Sections 2 and 3).  Defaults from sipg_default_params. */
typedef struct {
  int degree;              /* k = p in the paper, 1..8                         */
  double penalty_factor;   /* multiplies tau_e = (k+1)^2 A/V (Section 2); 1.0  */
  int precision;           /* V-cycle precision: 0 FP64, 1 FP32 (Section 4,
                              mixed-precision multigrid); the outer solver and
                              the coarse solve are always FP64              */
  int p_coarsen;           /* p-sequence of the FE levels (Section 3.2):
                              0 p_{l-1} = floor(p_l/2) (default, preferred by
                              the paper), 1 p_{l-1} = p_l - 1, 2 straight to 1 */
  int cheb_degree;         /* n_s smoothing steps pre and post, default 5      */
  double cheb_lo, cheb_hi; /* smoothing range [lo, hi] * lambda_max: 0.06, 1.2 */
  int eig_iters;           /* CG iterations of the lambda_max estimate, 20     */
  double lambda_override;  /* > 0: use this lambda_max on every level (tests)  */
  int smoother;            /* 0: Chebyshev-Jacobi (Algorithm 3)               */
  int operator_only;       /* 1: build only the finest DG operator (for
                              operator_apply); the solver calls then fail   */
  char coarsening[8];      /* order of the coarsening steps from the finest
                              level (Section 3.2, Table SummaryCoarsening-
                              Strategies): 'c' DG -> FE at equal h and p, 'p'
                              polynomial levels down to 1, 'h' geometric
                              levels; default "cph"; must contain 'c' and 'p'
                              (the dense coarse solve works on FE_1)       */
  int autotune;            /* 1: at setup, time a few tile shapes (cells per
                              thread block) of every cell kernel of every
                              level (both DG passes, the FE cell pass) in
                              both precisions and keep the fastest; the
                              candidates are the widths whose last wave of
                              blocks leaves the fewest cell slots idle;
                              cached per (degree, geometry, cells) for the
                              process                                      */
  int fe_assemble;         /* FE levels of degree <= fe_assemble (0..3;
                              default 1) apply an assembled (2p+1)^3-point
                              stencil built at setup from the same element
                              integrals instead of the matrix-free cell and
                              node passes (27 points at degree 1: one
                              node-centric launch instead of two); 0 = all
                              levels matrix-free.  Degrees 2 and 3 (125 and
                              343 points) are slower than matrix-free on
                              GB300 except on the smallest meshes and are
                              kept for comparison only                     */
  int coarse_dense_max;    /* coarsest level solved by a dense inverse up to
                              this many unknowns (default 2197 = 13^3 nodes:
                              every mesh whose sizes halve down to <= 12
                              cells); larger coarse levels (odd or prime
                              mesh sizes) are solved inexactly by the solver
                              that coarse_solver names, which the flexible
                              CG absorbs                                     */
  int coarse_iters;        /* Jacobi-PCG iterations (coarse_solver 1), 50      */
  int coarse_solver;       /* above coarse_dense_max (Section 3.3, "Coarse-
                              grid solver"): 0 CG preconditioned by one
                              smoothed-aggregation AMG V-cycle to
                              coarse_rtol (default, the paper's coarse
                              solver); 1 coarse_iters Jacobi-PCG iterations  */
  double coarse_rtol;      /* relative residual of the AMG-CG, 1e-3            */
  int coarse_maxit;        /* AMG-CG iterations launched per coarse solve
                              (each one skips its work once coarse_rtol is
                              met, so the solve stays capturable), 12       */
  int fuse_tail;           /* 1 (default): the V-cycle below the assembled
                              degree-1 levels of at most 8192 nodes (their
                              Chebyshev steps, residuals and 2:1 transfers,
                              Algorithms 2 and 3) and a dense coarse solve of
                              at most 1000 unknowns run as one launch of one
                              thread-block cluster, barriers between the
                              steps, with the same arithmetic as the
                              per-step launches (same results, bit for bit);
                              0: one launch per step                        */
  void *stream;            /* cudaStream_t or NULL                             */
} sipg_params;

typedef struct {
  int iterations;          /* outer iterations performed                       */
  int converged;           /* 1 if ||r||/||r0|| <= rtol was reached            */
  double r0_norm;          /* ||b - A x0||_2                                   */
  double r_norm;           /* final ||r||_2                                    */
  double rho;              /* average convergence rate (Section 5.1)           */
  double n10;              /* -10 / log10(rho)                                 */
  double seconds;          /* wall time of the solve on the stream             */
  double res_history[256]; /* ||r_j||_2, j = 0..min(iterations,255)            */
  int learned;             /* 1 if the solve started with the learned smoother */
  int fell_back;           /* 1 if it switched back to Chebyshev on the way    */
} sipg_solve_info;

/* Fills the defaults listed above (degree 3, FP64). */
void sipg_default_params(sipg_params *p);

/* Setup (Section 3.1: setup cost not part of the solve): 1D rules, geometry
 * and penalty per level, the cph level hierarchy (Section 3.2: DG_k -> FE_k ->
 * FE_floor(k/2) -> ... -> FE_1 -> FE_1 on coarser meshes while every m is even
 * and m/2 >= 3), transfer tables, inverse diagonals, lambda_max estimates by
 * eig_iters Jacobi-CG iterations, the dense coarse factor.  Allocates all
 * device memory of the context.  EINVAL for degree outside 1..8, m < 1,
 * non-positive extents, mapping_degree != 3 with deform, a penalty factor
 * <= 0, or no Dirichlet side when a solver will be used (the solver calls
 * then return EINVAL). */
sipg_status sipg_create(const sipg_mesh *mesh, const sipg_params *params, sipg_ctx **out);

/* Setup on an unstructured hexahedral mesh (see sipg_hex_mesh): the DG level
 * only (params->operator_only must be 1; the multigrid hierarchy needs the
 * box), for sipg_operator_apply, sipg_level_apply on level 0, sipg_time_apply
 * and the tile-shape calls.  DoF order: cell-major in the given cell order,
 * nodes of a cell lexicographic in its own reference coordinates (xi_0
 * fastest).  The operator is the one of Section 2 with tau_e from each cell's
 * own face areas and volume; on an interior face each side integrates with
 * its own geometry at the shared points.  EINVAL for vertex ids out of range,
 * a face shared by more than two cells, a singular cell map, or a face whose
 * corners match no symmetry of the square. */
sipg_status sipg_create_unstructured(const sipg_hex_mesh *mesh, const sipg_params *params, sipg_ctx **out);
sipg_status sipg_destroy(sipg_ctx *ctx);
const char *sipg_last_error(const sipg_ctx *ctx);

/* Number of levels (L+1) and the size of level l (0 = coarsest, L = finest DG). */
sipg_status sipg_num_levels(const sipg_ctx *ctx, int *nlevels);
sipg_status sipg_num_dofs(const sipg_ctx *ctx, int level, int64_t *n);
/* Level description: kind 0 = DG, 1 = FE; degree; cells per direction. */
sipg_status sipg_level_info(const sipg_ctx *ctx, int level, int *kind, int *degree, int m[3]);
/* lambda_max estimate of D^-1 A used by the smoother of level l (Section 3.1). */
sipg_status sipg_lambda(const sipg_ctx *ctx, int level, double *lambda);

/* Right-hand side of the manufactured solution (Section 5.3, cube): kind 0:
 * u = prod_j sin(pi (x_j - lo_j)/(hi_j - lo_j)), f = -lap u, g = u on the
 * Dirichlet sides (zero on the box), h = du/dn on Neumann sides.  Writes the
 * FP64 DG vector b_dev (length = dofs of the finest level). */
sipg_status sipg_rhs(sipg_ctx *ctx, int kind, double *b_dev);

/* L2 error || u_h - u ||_L2 of a finest-level FP64 solution against the
 * manufactured solution of sipg_rhs kind (0 only), with an (k+3)-point Gauss
 * rule per direction on the mapped cells; computed on the host (a diagnostic,
 * not part of the solve). */
sipg_status sipg_l2_error(sipg_ctx *ctx, int kind, const double *x_dev, double *err);

/* v = A u on the finest (DG) level: the homogeneous SIPG operator of
 * Eq. WeakFormDG with fluxes InteriorPenaltyFlux1/2 and mirror boundary
 * conditions, evaluated matrix-free by sum factorization (Section 4,
 * Eq. MatrixFreeAbstractNotation).  u and v must not overlap. */
sipg_status sipg_operator_apply(sipg_ctx *ctx, int precision, const void *u_dev, void *v_dev);

/* v = A_l u on any level (FE levels: Eq. WeakFormFE with constrained rows set
 * to the identity, Section 2), in either precision. */
sipg_status sipg_level_apply(sipg_ctx *ctx, int level, int precision, const void *u_dev, void *v_dev);

/* Inverse diagonal D^-1 of level l (Section 3.1), written in the level's
 * precision (finest level: precision argument). */
sipg_status sipg_inverse_diagonal(sipg_ctx *ctx, int level, int precision, void *d_dev);

/* nsteps Chebyshev-Jacobi steps of Algorithm 3 on A_l x = b, starting from
 * the given x (updated in place), in the level's V-cycle precision. */
sipg_status sipg_smooth(sipg_ctx *ctx, int level, const void *b_dev, void *x_dev, int nsteps);

/* Transfers between level l and l-1 (Section 3.2), V-cycle precision:
 * restrict:   rc = R r = P^T r   (r on level l, rc on level l-1)
 * prolongate: x += P xc          (xc on level l-1, x on level l)     */
sipg_status sipg_restrict(sipg_ctx *ctx, int level, const void *r_dev, void *rc_dev);
sipg_status sipg_prolongate_add(sipg_ctx *ctx, int level, const void *xc_dev, void *x_dev);

/* Coarse solve on level 0 in FP64 (Section 3.3, "Coarse-grid solver"): x =
 * A_0^-1 b by the dense inverse up to coarse_dense_max unknowns, above it the
 * inexact solve params.coarse_solver names (AMG-CG to coarse_rtol by default). */
sipg_status sipg_coarse_solve(sipg_ctx *ctx, const double *b_dev, double *x_dev);

/* What solves level 0: *kind = 0 dense inverse, 1 Jacobi-PCG, 2 AMG-CG; for
 * AMG-CG *nlevels AMG levels with sizes[0..min(nlevels,10)-1] rows (sizes[0]
 * = level 0's unknowns) and *last_iterations = CG iterations of the most
 * recent coarse solve on the context's stream (synchronizes that stream).
 * Any output pointer may be NULL. */
sipg_status sipg_coarse_info(sipg_ctx *ctx, int *kind, int *nlevels, int sizes[10], int *last_iterations);

/* One V-cycle of level 0's smoothed-aggregation AMG from x = 0 (Section 3.3):
 * x = M_AMG^-1 b, FP64 device vectors of level 0's length.  EINVAL unless
 * level 0 is solved by AMG-CG. */
sipg_status sipg_coarse_amg_vcycle(sipg_ctx *ctx, const double *b_dev, double *x_dev);

/* One V-cycle of Algorithm 2 with x = 0 on entry: z = M^-1 r.  r and z are
 * FP64 finest-level vectors; the cycle runs in params.precision. */
sipg_status sipg_vcycle(sipg_ctx *ctx, const double *r_dev, double *z_dev);

/* Solve A x = b (Algorithm 1 structure, flexible CG with one retained
 * direction) preconditioned by one V-cycle, FP64 residual and inner
 * products.  x_dev holds the start vector on entry.  Stops when
 * ||r||/||r0|| <= rtol or after maxit iterations; fixed_iters > 0 runs exactly
 * that many iterations instead.  info may be NULL.  ENOTCONV if maxit was
 * hit, EBREAKDOWN on p^T A p <= 0 or non-finite scalars, ENAN for a
 * non-finite right-hand side. */
sipg_status sipg_solve(sipg_ctx *ctx, const double *b_dev, double *x_dev, double rtol,
                       int maxit, int fixed_iters, sipg_solve_info *info);

/* Several right-hand sides of the context's problem solved together (not in
 * the paper, whose solver takes one right-hand side per run): B_dev and
 * X_dev hold nrhs device vectors of num_dofs values one after another (vector
 * r at r * num_dofs, the oracle's DoF order in each), X_dev is the initial
 * guess and the result.  One flexible CG per right-hand side, all in lockstep:
 * every operator application and every V-cycle runs on all nrhs vectors with
 * one launch per kernel (block b of a cell kernel = cell group b / nrhs of
 * vector b % nrhs, so the vectors share each group's geometry reads).  Each
 * right-hand side stops on its own at rtol (or maxit); the iterates of each
 * equal those of sipg_solve on it alone up to rounding.  infos: nrhs entries
 * (may be NULL).  1 <= nrhs <= 4096; device memory for nrhs vectors of every
 * level is allocated on first use and kept.  Errors: EINVAL, ENAN (a right-hand
 * side not finite), ENOTCONV, EBREAKDOWN as for sipg_solve. */
sipg_status sipg_solve_multi(sipg_ctx *ctx, int nrhs, const double *B_dev, double *X_dev, double rtol, int maxit,
                             sipg_solve_info *infos);

/* V = A U for nv vectors at once (same layout as sipg_solve_multi), in the
 * given precision (0 FP64, 1 FP32); the same kernels as sipg_operator_apply
 * with one launch per pass for all vectors.  Needs a solver context. */
sipg_status sipg_operator_apply_multi(sipg_ctx *ctx, int precision, int nv, const void *U_dev, void *V_dev);

/* The same solve from and to HOST memory: copies b_host to the device, solves
 * with x0 = 0, copies x back to x_host (both FP64, length = finest dofs). */
sipg_status sipg_solve_host(sipg_ctx *ctx, const double *b_host, double *x_host, double rtol,
                            int maxit, sipg_solve_info *info);

/* Per-launch device time of the last sipg_operator_apply-style launches
 * recorded with events on the context stream: the DG evaluation pass and the
 * DG integration pass, in milliseconds (for roofline accounting). */
sipg_status sipg_time_apply(sipg_ctx *ctx, int precision, const void *u_dev, void *v_dev,
                            int repeats, float *ms_eval, float *ms_integrate);

/* ---- Many problems at once (not in the paper, whose solver handles one
 * problem per run; each problem's method is unchanged).  A batch holds nprob
 * independent problems -- uneven meshes and degrees, or the same mesh repeated
 * for many right-hand sides.  meshes[i], params[i] describe problem i (all
 * affine or all curved; one precision for all; each needs a Dirichlet side);
 * params[0].stream is the stream of the batched work.  The finest-level
 * operators of all problems run as one persistent launch per pass (a fixed
 * grid walking a work list of (problem, cell block) items, longest first);
 * the flexible-CG iterations run in lockstep with batched inner products and
 * updates (blocks per problem in proportion to its size).  On a non-default
 * stream, when every problem's hierarchy starts with a DG level above a
 * matrix-free FE level of the same degree (cph), the V-cycles of all problems
 * are one captured graph: the Chebyshev steps, residuals and c-transfers of
 * those two levels are shared batched launches over all problems; below them
 * each problem's own cycle is a branch of the graph; a problem of 2^21 DoF or
 * more keeps its whole cycle as a branch beside the shared launches.  The
 * lockstep iteration then runs in captured chunks gated on the device (one
 * host read per chunk).  Otherwise each problem's V-cycle (a CUDA graph) runs
 * on its own stream and the host reads the scalars every iteration.  Every
 * problem's numbers are those of its own single-problem kernels either way. */
typedef struct sipg_batch sipg_batch;
sipg_status sipg_batch_create(int nprob, const sipg_mesh *meshes, const sipg_params *params, sipg_batch **out);
sipg_status sipg_batch_destroy(sipg_batch *batch);
const char *sipg_batch_last_error(const sipg_batch *batch);
/* The context of problem i (owned by the batch; do not destroy it). */
sipg_status sipg_batch_context(sipg_batch *batch, int i, sipg_ctx **ctx);
/* v[i] = A_i u[i] (FP64, finest level) for every problem: two launches total. */
sipg_status sipg_batch_apply(sipg_batch *batch, const double *const *u_dev, double *const *v_dev);
/* z[i] = M_i^-1 r[i] (FP64 in and out): one V-cycle (Algorithm 2) of every
 * problem, through the batched cycle where it applies (above).  Each z[i]
 * equals sipg_vcycle on problem i's context bit for bit.  EINVAL for a NULL
 * array or entry. */
sipg_status sipg_batch_vcycle(sipg_batch *batch, const double *const *r_dev, double *const *z_dev);
/* Solve A_i x[i] = b[i] for every problem to ||r||/||r0|| <= rtol (x[i] holds
 * the start vector); infos (array of nprob, may be NULL) gets each problem's
 * history.  Status as sipg_solve, worst over the problems. */
sipg_status sipg_batch_solve(sipg_batch *batch, const double *const *b_dev, double *const *x_dev, double rtol,
                             int maxit, sipg_solve_info *infos);

/* ---- Learned smoother (not in the paper).  A per-cell network stands in for
 * the Chebyshev smoother on the finest level: input = the cell's (k+1)^3
 * residual values followed by, per face (-x,+x,-y,+y,-z,+z), the neighbour's
 * (k+1)^2 residual values on the shared face (zeros on the boundary), all
 * divided by their RMS s; two hidden ReLU layers of width 256; output y of
 * (k+1)^3 values; smoothing step x <- x + c s y per cell.  BF16 weights and
 * activations, FP32 accumulation (tensor cores), FP32 master weights.  The
 * solve stays a flexible CG, so its result does not depend on the network;
 * the Chebyshev cycle's average rate rho (measured while generating the data)
 * judges each learned step by residual reduction per unit time: a step that
 * reduces the residual by less than rho^(t_learned / t_chebyshev), with t the
 * time of one iteration with each cycle (measured after training), switches
 * the solve back to Chebyshev (sipg_solve_info.fell_back). */
typedef struct {
  int npairs, epochs, steps;      /* training pairs, epochs, Adam steps          */
  double loss_first, loss_last;   /* mean squared error, first and last epoch    */
  double out_scale;               /* c                                            */
  double cheb_rate;               /* average rate of the Chebyshev cycle         */
  double seconds;                 /* wall time of data generation and training  */
  double target_max;              /* largest |e|/s of the data (before scaling)  */
  double nonfinite;               /* number of non-finite targets (0 expected)   */
  double iter_ms_chebyshev;       /* one flexible-CG iteration's V-cycle plus    */
  double iter_ms_learned;         /* outer apply, with each smoother (ms)        */
  double damping;                 /* omega applied to c after training           */
  double step_reduction;          /* ||r - omega A d|| / ||r|| of that step      */
} sipg_train_info;
/* Generates npairs (cell residual -> cell error) pairs from the plain cycle
 * and trains the network with Adam (batches of 256).  For the first 4
 * flexible-CG iterates of 4 seeded uniform right-hand sides, the cycle's input
 * b_v = r_j and its exact correction x* = A^-1 b_v (solved to 1e-12) give
 * pairs at seeded random cells after pre-smoothing and the coarse-grid
 * correction (b_v - A x, x* - x): the high-frequency error a smoother works
 * on.  Then the step is damped: on the last such residual r the output scale
 * c is multiplied by the omega minimising ||r - omega A d|| for the step d
 * taken from x = 0. */
sipg_status sipg_smoother_train(sipg_ctx *ctx, int npairs, int epochs, uint64_t seed, sipg_train_info *info);
/* Fine-tune the trained network in the energy norm (not in the paper): on
 * the full-mesh snapshots kept by sipg_smoother_train (residual r and error e
 * of the state the post-smoother starts from; 16 of them) minimise
 * ||e - d||_A^2 / ||e||_A^2 for the step d = c s net(features(r)) of all cells
 * (its gradient -2 (r - A d) / e.r: one operator application per step), Adam
 * with learning rate lr (0: 3e-4), `epochs` passes over the snapshots; the
 * Adam moments restart at every call, so calls accumulate passes; then damp the
 * step by the energy-optimal omega = d.r / d.A d on the last snapshot.  info
 * (may be NULL): loss before/after (mean over the snapshots of the first and
 * the last pass), steps, seconds, damping.  EINVAL before training, for
 * epochs outside 1..100000 or lr outside [0, 1]; ENAN if the loss stops being
 * finite. */
sipg_status sipg_smoother_finetune(sipg_ctx *ctx, int epochs, double lr, sipg_train_info *info);

/* which = 0: Chebyshev (default); 1: learned (trained network required), with
 * steps_pre and steps_post network steps around the coarse correction; 2: the
 * same learned cycle without the Chebyshev fallback (to measure the network
 * alone: the flexible CG still returns a correct result, or stops at maxit);
 * steps_pre = 0 keeps Chebyshev pre-smoothing (the network is trained on the
 * post-smoothing state), 1..16 network steps; steps_post 0..16, where 0
 * leaves the finest level without post-smoothing (the cycle without the
 * network, to measure what its steps add).  Selecting the learned smoother
 * with new step counts times one solver iteration of that cycle (a few
 * V-cycles on the context's stream, synchronised) for the fallback test. */
sipg_status sipg_set_smoother(sipg_ctx *ctx, int which, int steps_pre, int steps_post);
/* Network shape: in_dim (and padded width), hidden width, out_dim (and
 * padded width), number of parameters.  Flat parameter layout (FP32):
 * W1[in_pad][hidden], b1[hidden], W2[hidden][hidden], b2[hidden],
 * W3[hidden][out_pad], b3[out_pad]. */
sipg_status sipg_mlp_shape(sipg_ctx *ctx, int *in_dim, int *in_pad, int *hidden, int *out_dim, int *out_pad,
                           int64_t *nparams);
/* set = 1: load the parameters from host; 0: store them to host. */
sipg_status sipg_mlp_params(sipg_ctx *ctx, int set, float *host);
/* Y[B][out_pad] = network(X[B][in_dim]) (device FP32 arrays). */
sipg_status sipg_mlp_forward(sipg_ctx *ctx, const float *X_dev, int B, float *Y_dev);
/* Gradients of sum ||y - t||^2 / (2B) over B rows (X[B][in_dim], T[B][out_dim],
 * device) to host (flat layout), and the loss. */
sipg_status sipg_mlp_gradients(sipg_ctx *ctx, const float *X_dev, const float *T_dev, int B, float *grads_host,
                               double *loss);
/* Network inputs of every cell from a finest-level FP64 residual: feat[cells][in_pad]
 * (already divided by s, BF16-rounded) and scale[cells] = s. */
sipg_status sipg_mlp_features(sipg_ctx *ctx, const double *r_dev, float *feat_dev, float *scale_dev);

/* Cells per thread block a cell kernel of a level uses in the given
 * precision (pass 0 DG evaluation, 1 DG integration on a DG level; 2 the FE
 * cell pass on an FE level): the autotuned or set value, else the default
 * (about 256 threads per block, fewer cells per block on meshes that would
 * otherwise give fewer blocks than the GPU has SMs).  EINVAL for a pass that
 * does not exist on the level. */
sipg_status sipg_tile_shape(const sipg_ctx *ctx, int level, int precision, int pass, int *cells_per_block);

/* Sets that width (0 = the default above; at most 768 threads and 227 KB
 * of shared memory per block, else EINVAL).  The results do not depend on
 * it: every cell is computed by the same threads in the same order.  Drops
 * the context's captured V-cycle graphs (they hold the old launch shapes). */
sipg_status sipg_set_tile_shape(sipg_ctx *ctx, int level, int precision, int pass, int cells_per_block);

/* Number of kernels the library has launched in this process so far, all
 * contexts together: a kernel inside a replayed CUDA graph counts once per
 * replay (in a graph of conditional nodes, only the bodies that ran); a
 * capture itself launches nothing.  For launch accounting. */
sipg_status sipg_launch_count(unsigned long long *n);

/* Peak arithmetic probe: runs an independent-FMA loop on every SM for the
 * given precision (0 FP64 DFMA, 1 FP32 FFMA, 2 FP64 tensor-core mma.sync
 * m8n8k4) and returns the measured rate in FLOP/s (2 per multiply-add).  Not
 * part of the method: used for the roofline.  EINVAL for another value. */
sipg_status sipg_fma_peak(int precision, void *stream, double *flops_per_s);

/* Operator apply that allocates no device memory.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc when
 * they need A u -- for example code inside a framework whose caching allocator
 * already holds the GPU's memory, or a time-stepping loop that must not
 * allocate once it runs.  Computes v = A u, the same FP64 operator as
 * sipg_operator_apply for affine cells (mesh->deform must be 0), with
 * penalty_factor as in sipg_params.  The caller passes the device vectors u
 * and v (length m0 m1 m2 (degree+1)^3, DG order; overlapping ranges are
 * rejected with SIPG_EINVAL); every
 * other buffer lives in one static device array of 64 MiB that each GPU
 * loading the library holds until the process exits.  Problems whose scratch
 * (3 (k+1)^3 + 12 (k+1)^2 + 1 doubles per cell, plus small tables) exceeds
 * 64 MiB are rejected with SIPG_EINVAL (about 1.4 million DoF at degree 3).
 * The first call on a device looks up the array's device address and uploads
 * the 1D tables (both synchronous); make that first call before any stream
 * capture.  All calls share the one array: two calls whose work overlaps on
 * the GPU (different streams, or different host threads) race and give wrong
 * results; calls ordered on one stream are safe.  Nothing in the array needs
 * to start at zero (every call rewrites what it reads).  Work is queued on
 * `stream` (cudaStream_t, NULL = legacy default stream); on failure
 * sipg_last_error(NULL) describes it.  A CUDA error left pending by the
 * caller's earlier work is cleared on entry (cudaGetLastError), so that it is
 * not reported as this call's failure. */
sipg_status sipg_operator_apply_noalloc(const sipg_mesh *mesh, int degree, double penalty_factor,
                                        const double *u_dev, double *v_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif
