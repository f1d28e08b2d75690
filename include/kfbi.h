/*
 * kfbi.h — C ABI of the GB300 correction-function KFBI library.
 *
 * The library evaluates the boundary integral operators of the kernel-free
 * boundary integral method of Zhou & Ying, "A correction function-based
 * kernel-free boundary integral method for elliptic PDEs with implicitly
 * defined interfaces" (arXiv 2309.05965), and solves the resulting boundary
 * integral equations with matrix-free GMRES, entirely on one GPU.
 *
 * Conventions (all entry points):
 *   - Every array argument is a DEVICE pointer unless stated otherwise; the
 *     caller owns it and keeps it alive until the enqueued work has finished.
 *   - Work is enqueued on the CUDA stream given to kfbi_create_problem.  Calls
 *     return after enqueueing, except where a host-visible result is produced
 *     (kfbi_create_problem, kfbi_gmres_solve, size queries), which synchronise
 *     that stream.
 *   - Grids are (N+1)^d FP64 node arrays over the box [lo, hi]^d, C order with
 *     the last axis fastest: node (i0, i1[, i2]) has linear index
 *     (i0 (N+1) + i1) (N+1) + i2 and coordinates lo + i_k h, h = (hi - lo)/N.
 *   - DOF arrays (length N_b) follow the DOF order: family r ascending (the
 *     point lies on a grid line parallel to e_r), then the grid line (other
 *     axes lexicographic, lower axis slowest), then the position along it.
 *   - Sign conventions (Sec. 2, Sec. 5): Omega = {H < 0} is the '+' side; the
 *     normal n = grad H / |grad H| points out of Omega; jumps are
 *     [v] = v(inside) - v(outside).
 *   - No call throws; every call returns a kfbi_status, and kfbi_last_error
 *     returns a message for the last failure on that problem.
 *   - There is no CPU fallback: a build without a usable GPU fails at create.
 */
#ifndef KFBI_H
#define KFBI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KFBI_OK = 0,
  KFBI_ERR_ARG = 1,            /* invalid argument or size                       */
  KFBI_ERR_GEOMETRY = 2,       /* no collocation stencil (under-resolved Gamma)  */
  KFBI_ERR_SINGULAR = 3,       /* collocation / trace system singular (cond>1e10)*/
  KFBI_ERR_NOT_CONVERGED = 4,  /* GMRES or inner box solve reached its limit     */
  KFBI_ERR_NONFINITE = 5,      /* NaN or Inf in data or results                  */
  KFBI_ERR_TIMEOUT = 6,        /* a bounded device wait gave up                  */
  KFBI_ERR_CUDA = 7,           /* a CUDA runtime call failed                     */
  KFBI_ERR_UNSUPPORTED = 8     /* configuration not supported                    */
} kfbi_status;

/* Analytic level-set families H (Sec. 5.1: Gamma = {H = 0}). */
typedef enum {
  KFBI_LS_ELLIPSE = 1,    /* 2D p=[cx,cy,a,b,theta]: rotated ellipse              */
  KFBI_LS_STAR = 2,       /* 2D p=[cx,cy,R0,A,k]: r - R0 - A sin(k theta)         */
  KFBI_LS_ELLIPSOID = 3,  /* 3D p=[cx,cy,cz,a,b,c]                                */
  KFBI_LS_TORUS = 4,      /* 3D p=[R,r]: (sqrt(x^2+y^2)-R)^2 + z^2 - r^2          */
  KFBI_LS_MOLECULE = 5,   /* 3D p=[r,level,n,x1,y1,z1,...]: level - sum exp(-|x-x_k|^2/r^2) */
  KFBI_LS_DISCS = 6,      /* 2D p=[r,n,x1,y1,...]: min_k |x-x_k|^2 - r^2, n discs, one
                             interface each (close or touching allowed)          */
  KFBI_LS_SPHERES = 7,    /* 3D p=[r,n,x1,y1,z1,...]: the same with balls          */
  KFBI_LS_GRID = 8,       /* 2D or 3D: H known only by its values at the (N+1)^d
                             nodes of the problem's grid (kfbi_levelset.samples, a
                             sampled signed distance or any smooth level-set
                             function); between nodes H is the tensor-product
                             cubic Lagrange interpolant on the 4^d nodes around
                             the point (its cell clamped to [1, N-2] per axis;
                             a coordinate within 1e-10 h of a node is that
                             node, so H at a node is its sample); every
                             sample must be finite (KFBI_ERR_ARG otherwise,
                             at create or update); p unused                   */
  KFBI_LS_UNION = 9       /* 2D or 3D p=[m, kind_1, params_1..., kind_2, ...]: m
                             interfaces, each of kind ELLIPSE or STAR (5
                             params) in 2D, ELLIPSOID (6) or TORUS (2) in 3D,
                             with its own function H_k; Omega = union of the
                             {H_k < 0}                                         */
} kfbi_levelset_kind;

/* Several interfaces (KFBI_LS_DISCS, KFBI_LS_SPHERES, KFBI_LS_UNION; the remark
 * on arbitrarily close interfaces in Sec. 5.2).  Interface k bounds the
 * component Omega^(k) = {H_k < 0}; every grid node carries a side label, 0
 * outside Omega and 1 + k in Omega^(k) (a node inside two overlapping
 * components: the first k with the smallest H_k).  Interfaces may be closer
 * than the grid step or touch: a grid edge whose end nodes carry labels a != b
 * holds one DOF on interface a - 1 (if a > 0) and one on b - 1 (if b > 0),
 * each where that H_k changes sign, the first node's first.  Each interface
 * has its own correction function C^(k) = u^(k) - u^(0) (Omega^(0) = outside),
 * fitted from the DOFs of interface k only; a stencil joining labels l_P and
 * l_Q is corrected with C^(l_P)(Q) - C^(l_Q)(Q) (C^(0) = 0).  Jump data g1, g2
 * at a DOF are those of its own interface (kfbi_dof_iface).  At most 32
 * interfaces. */
#define KFBI_MAX_INTERFACES 32

typedef enum {
  KFBI_DIRICHLET_INTERIOR = 0, /* eq. (bie-D): (1/2 + K) phi = g_D - G f           */
  KFBI_INTERFACE_MU = 1,       /* mu-form BIE of Sec. 3.2 for psi = [d_n u]         */
  KFBI_NEUMANN_INTERIOR = 2,   /* eq. (bie-N): (1/2 - K') psi = g_N - sigma d_n G f;
                                  kappa = 0: projected to zero mean (Sec. 7.2.1)    */
  KFBI_INTERFACE_GENERAL = 3   /* eq. (bie-ifp-1): any sigma_i, kappa_i; unknowns
                                  [phi; psi] = [u_1; sigma_2 d_n u_2], 2 N_b values */
} kfbi_problem_kind;

typedef enum { KFBI_BOX_DST = 0, KFBI_BOX_MG = 1 } kfbi_box_solver;
typedef enum { KFBI_FP64 = 0, KFBI_MIXED = 1 } kfbi_precision;

#define KFBI_LS_MAX_PARAMS 64

typedef struct {
  int kind;                      /* kfbi_levelset_kind */
  int n_params;
  double p[KFBI_LS_MAX_PARAMS];
  const double* samples;         /* KFBI_LS_GRID: device array of the (N+1)^d node
                                    values in grid order, copied at create (the
                                    caller may free it afterwards); NULL otherwise */
} kfbi_levelset;

typedef struct {
  int dim;                /* 2 or 3                                               */
  int n;                  /* intervals per axis N, a power of two: DST box solve
                             2D 8..2048 (FP64) / 8..4096 (mixed), 3D 8..1024
                             within device memory; multigrid from 8.  Larger
                             sizes: KFBI_ERR_UNSUPPORTED at create          */
  double lo, hi;          /* box [lo, hi]^dim                                     */
  int order;              /* 4 (compact 9/27-point) or 2 (5/7-point)              */
  int kind;               /* kfbi_problem_kind                                    */
  double sigma_in;        /* sigma in Omega (the '+' side)                         */
  double sigma_out;       /* sigma outside (interface problem only)               */
  double kappa;           /* Dirichlet BVP: kappa of eq. (BVP); mu-form: kappa~ of
                             eq. (bie-ifp-2) (kappa_i / sigma_i, the same on both
                             sides)                                               */
  int box_solver;         /* kfbi_box_solver                                      */
  int precision;          /* kfbi_precision: FP64, or FP32 box solve with FP64
                             residuals and iterative refinement                   */
  double cos_alpha;       /* overlapping surface decomposition; <= 0 selects the
                             default (0.707 in 2D, 0.4 in 3D)                     */
  double box_rtol;        /* inner tolerance of MG / refinement (<= 0: 1e-13)     */
  int box_max_iters;      /* inner iteration limit (<= 0: 60)                     */
  double kappa_out;       /* general interface problem: kappa_2 of Omega_2 (kappa
                             is then kappa_1 of Omega_1); unused otherwise        */
  double relax;           /* inexact GMRES (mixed-precision box solves, sine
                             transform or multigrid): 0 = every operator
                             application refined to box_rtol; omega in (0, 1] =
                             before application j inside kfbi_gmres_solve the
                             refinement stops at max(box_rtol, omega rtol ||b|| /
                             ||r_j||) (relaxation as the residual falls, after
                             Simoncini & Szyld 2003); right-hand side, starts,
                             restarts and evaluation stay at box_rtol           */
} kfbi_config;

/* Problem data (Sec. 2).  f_* are the physical right-hand sides f of eqs.
 * (BVP)/(IFP) on each side, smoothly extended to the whole box; the library
 * divides them by sigma.  lapf_* are their Laplacians (for the h^2/12 Lap f term
 * of eqs. (9p-cds)/(27p-cds)).  Dirichlet BVP: g1 = g_D, g2, f_out, lapf_out and
 * g_b unused (may be NULL).  Neumann BVP: g2 = g_N = sigma d_n u, g1, f_out,
 * lapf_out and g_b unused (may be NULL).  Interface: g1 = [u], g2 = [sigma d_n u], g_b = outer
 * Dirichlet values (NULL = homogeneous).  Any grid may be NULL (= 0). */
typedef struct {
  const double* g1;       /* N_b   */
  const double* g2;       /* N_b   */
  const double* f_in;     /* grid  */
  const double* f_out;    /* grid  */
  const double* lapf_in;  /* grid  */
  const double* lapf_out; /* grid  */
  const double* g_b;      /* grid (only its box-boundary layer is read) */
  int in_per_interface;   /* 0: f_in and lapf_in are one grid for every
                             interface; 1 (several interfaces): each holds one
                             grid per interface, consecutive, grid k the f of
                             Omega^(k) smoothly extended to the whole box     */
} kfbi_data;

typedef struct {
  double rtol;            /* stop at ||b - A x|| <= rtol ||b||                     */
  int restart;            /* Krylov dimension before a restart (<= 100)           */
  int max_iter;           /* total operator applications                          */
  const double* x0;       /* initial density (device, N_b) or NULL for zero       */
} kfbi_gmres_opts;

typedef struct {
  int iters;              /* operator applications in Arnoldi                     */
  double rel_res;         /* final ||b - A x|| / ||b|| (GMRES estimate)           */
  double t_ms[8];         /* [0] BIE right-hand side, [1] GMRES loop, [2] total   */
  int x0_rejected;        /* 1 if opts->x0 was given but its residual was not
                             below ||b||, so GMRES started from zero instead    */
  int refine_steps;       /* mixed DST box solves: the FP32 correction steps run
                             during the call beyond each box solve's first FP32
                             solve (both operators for the general kind); 0
                             otherwise                                          */
} kfbi_gmres_info;

typedef struct kfbi_problem kfbi_problem;

/* Kernel classes for launch accounting and profiling (kfbi_profile_*). */
typedef enum {
  KFBI_KC_CORRECTION = 0,  /* C at irregular nodes (Step 3.1)                  */
  KFBI_KC_RHS = 1,         /* corrected right-hand side (Step 3.2)             */
  KFBI_KC_DST = 2,         /* sine-transform passes of the box solve (3.3)     */
  KFBI_KC_RESIDUAL = 3,    /* FP64 residual / norms of the refinement (3.3)    */
  KFBI_KC_MG = 4,          /* multigrid smoothing and transfers (3.3)          */
  KFBI_KC_TRACE = 5,       /* corrected interpolation + BIE combination (3.4)  */
  KFBI_KC_GMRES = 6,       /* Arnoldi, Givens and updates (Step 4)             */
  KFBI_KC_OTHER = 7,
  KFBI_KC_COUNT = 8
} kfbi_kernel_class;

/* ---- problem lifetime -------------------------------------------------- */

/* Builds the discretisation of one geometry on the GPU (Sec. 5.1, 5.4):
 * node classes, grid-line intersections (the DOFs), reference planes,
 * collocation stencils and the inverses of the collocation matrices M (eq.
 * (cau-ls)), irregular nodes and their closest primary points, the correction
 * stencils (eq. (crc-formula)), the trace least-squares weights (Sec. 5.5) and
 * the box solver.  `cuda_stream` is a cudaStream_t (NULL = legacy default).
 * On failure *out is NULL; KFBI_ERR_GEOMETRY / KFBI_ERR_SINGULAR report an
 * under-resolved interface. */
kfbi_status kfbi_create_problem(const kfbi_config* cfg, const kfbi_levelset* ls,
                                void* cuda_stream, kfbi_problem** out);
kfbi_status kfbi_destroy_problem(kfbi_problem* p);
/* A new interface on the same grid and configuration (a moving interface: the
 * level-set method of the paper's closing remarks, one set-up per time step):
 * the geometry, stencils, correction entries, trace weights and GMRES
 * workspace are rebuilt as kfbi_create_problem builds them, while the box
 * solver, its grids and the streams are kept.  N_b and every size query may
 * change; densities and starts of the old interface do not apply to the new
 * one.  The problem must not belong to a batch.  On failure the problem
 * holds no interface: update it again or destroy it.  Synchronises the
 * stream. */
kfbi_status kfbi_update_levelset(kfbi_problem* p, const kfbi_levelset* ls);
/* Message of the last failure on p; with p == NULL, of the last failed
 * kfbi_create_problem on the calling thread.  Owned by the library. */
const char* kfbi_last_error(const kfbi_problem* p);

/* ---- sizes and geometry queries ---------------------------------------- */

/* N_b, number of irregular nodes, and the number of polynomial coefficients
 * per primary point (15/35 for p = 4, 6/10 for p = 2). Host outputs. */
kfbi_status kfbi_sizes(const kfbi_problem* p, int* n_b, int* n_irr, int* n_coef);
kfbi_status kfbi_num_dofs(const kfbi_problem* p, int* n_b);
/* DOF coordinates and unit normals, (N_b, dim) row-major. */
kfbi_status kfbi_dof_points(const kfbi_problem* p, double* xyz, double* normals);
/* Per DOF: family r, reference axis argmax|n_k|, axis used by its stencil. */
kfbi_status kfbi_dof_info(const kfbi_problem* p, int32_t* family, int32_t* axis,
                          int32_t* stencil_axis);
/* Collocation stencils (Sec. 5.4): PDE node linear indices (N_b, n_pde),
 * Dirichlet DOF indices (N_b, n_dir), Neumann DOF indices (N_b, n_neu). */
kfbi_status kfbi_stencil_sizes(const kfbi_problem* p, int* n_pde, int* n_dir, int* n_neu);
kfbi_status kfbi_collocation_stencils(const kfbi_problem* p, int32_t* pde_nodes,
                                      int32_t* dir_dofs, int32_t* neu_dofs);
/* Node side labels, one byte per grid node: 0 outside Omega, 1 inside (one
 * interface), 1 + k in Omega^(k) (several interfaces). */
kfbi_status kfbi_inside_mask(const kfbi_problem* p, uint8_t* mask);
/* Irregular nodes I_h (a node of another label in the stencil) in
 * linear-index order and, with one interface, the closest primary point of
 * each (Sec. 5.3 partition of unity); with several interfaces owner must be
 * NULL (see kfbi_correction_entries). */
kfbi_status kfbi_irregular_nodes(const kfbi_problem* p, int32_t* lin_index, int32_t* owner);
/* Number of interfaces and of correction entries (the values of
 * kfbi_correction_values).  One interface: one entry per irregular node. */
kfbi_status kfbi_interfaces(const kfbi_problem* p, int* n_iface, int* n_entries);
/* Per DOF: the interface it lies on (device, N_b). */
kfbi_status kfbi_dof_iface(const kfbi_problem* p, int32_t* iface);
/* Correction entries (node, interface k) holding C^(k), in node order then k
 * (device arrays of n_entries): every irregular node for each k + 1 among the
 * labels of its stencil, and, near another interface, the nodes the trace fits
 * use (Sec. 5.5); owner = the closest primary point on interface k. */
kfbi_status kfbi_correction_entries(const kfbi_problem* p, int32_t* lin_index, int32_t* iface,
                                    int32_t* owner);

/* ---- the four steps of Algorithm 1, Step 3, one at a time -------------- */

/* Step 3.1: coefficients d_i of every local correction polynomial (N_b, n_coef),
 * graded-lexicographic monomial order in xi = (x - p_i)/h.  a = [u], b = [d_n u]
 * at the DOFs; ftilde = f~ = f+/sigma - f-/sigma grid (NULL = 0). */
kfbi_status kfbi_collocation_fit(kfbi_problem* p, const double* a, const double* b,
                                 const double* ftilde, double* coef);
/* Correction function C_h at every correction entry (n_entries; one
 * interface: the irregular nodes), eq. (local-cau-prb) with the closest-point
 * partition of unity.  ftilde: one grid for every interface. */
kfbi_status kfbi_correction_values(kfbi_problem* p, const double* a, const double* b,
                                   const double* ftilde, double* cvals);
/* Step 3.2: right-hand side of eq. (corrected-FDS) on the grid: F + h^2/12 Lap F
 * from each node's own side (data may be NULL = no source), plus C_P of eq.
 * (crc-formula), minus the outer-boundary lift of data->g_b.  Boundary layer 0. */
kfbi_status kfbi_corrected_rhs(kfbi_problem* p, const double* cvals, const kfbi_data* data,
                               double* rhs);
/* Step 3.3: u = A_h^{-1} rhs on the interior (DST-I or multigrid, FP64 or
 * mixed precision, per the config); boundary layer of u set to 0. */
kfbi_status kfbi_box_solve(kfbi_problem* p, const double* rhs, double* u);
/* Diagnostics of the last box solve on p (Step 3.3; synchronises the stream;
 * host outputs, each may be NULL): steps = FP32 solves of the mixed sine
 * transform (the first plus every refinement step its convergence flag let
 * run; 1 for the FP64 transform), outer steps of the mixed multigrid or 1 for
 * the FP64 multigrid; cycles = V-cycles run (0 for the sine transform);
 * rel_change = the last measured correction max|delta u| / max|u| (mixed) or
 * normwise backward error (FP64 multigrid), 0 for the FP64 transform;
 * converged = 1 if the inner tolerance was met.  The counts are those of the
 * work that ran on the device, not of the launches enqueued. */
kfbi_status kfbi_box_solve_info(kfbi_problem* p, int* steps, int* cycles, double* rel_change,
                                int* converged);
/* Step 3.4: one-sided values and normal derivatives at every DOF from a grid
 * function u and C at the irregular nodes (Sec. 5.5).  Any output may be NULL. */
kfbi_status kfbi_traces(kfbi_problem* p, const double* u, const double* cvals,
                        double* val_plus, double* val_minus, double* dn_plus,
                        double* dn_minus);

/* ---- operators and solves ---------------------------------------------- */

/* One application of the discrete BIE operator (Steps 3.1-3.4 plus the BIE
 * combination).  x and y hold N_b values, or 2 N_b ([phi; psi]) for the
 * general interface problem, whose operator is the left-hand side of eq.
 * (bie-ifp-1): with w_i the potential of box operator Lap - kappa_i/sigma_i
 * and jumps [u] = phi, [d_n u] = psi/sigma_i, y = [phi - (avg w_1 - avg w_2);
 * psi - (sigma_1 avg d_n w_1 - sigma_2 avg d_n w_2)] (two box solves).
 * Dirichlet y = x/2 + avg trace of D x; mu-form
 * y = x/2 - mu avg d_n of (-S x); Neumann y = x/2 + avg d_n of (-S x), for
 * kappa = 0 minus its arithmetic mean over the DOFs (Sec. 7.2.1: the solution
 * is fixed up to a constant; the right-hand side is projected the same way). */
kfbi_status kfbi_apply_operator(kfbi_problem* p, const double* x, double* y);
/* Right-hand side of the BIE (Algorithm 1, Step 1): N_b values, 2 N_b for
 * the general interface problem (the right-hand side of eq. (bie-ifp-1)). */
kfbi_status kfbi_bie_rhs(kfbi_problem* p, const kfbi_data* data, double* b);
/* Algorithm 1: BIE right-hand side, GMRES (Step 4) from opts->x0 or zero.
 * A given x0 whose residual ||b - A x0|| is not below ||b|| (or not finite)
 * is dropped and GMRES starts from zero (info->x0_rejected = 1): a learned or
 * otherwise approximate start can never make the solve worse than zero.
 * density: N_b output (2 N_b, [phi; psi], for the general interface problem;
 * opts->x0 likewise). info: host pointer (may be NULL). */
kfbi_status kfbi_gmres_solve(kfbi_problem* p, const kfbi_data* data,
                             const kfbi_gmres_opts* opts, double* density,
                             kfbi_gmres_info* info);
/* Grid solution from a density by superposition (one more potential solve):
 * Dirichlet u = D phi + N f; Neumann u = -S psi + N f (kappa = 0: up to an
 * additive constant); interface u with [u] = g1, [d_n u] = psi; general
 * interface problem: in Omega_1 the kappa_1 potential of [u] = phi,
 * [d_n u] = (psi + g2)/sigma_1, f_1; in Omega_2 the kappa_2 potential of
 * [u] = g1 - phi, [d_n u] = -psi/sigma_2, f_2 and g_b (two box solves). */
kfbi_status kfbi_evaluate(kfbi_problem* p, const kfbi_data* data, const double* density,
                          double* u_grid);

/* ---- batched solves ------------------------------------------------------ */

/* Many independent problems solved together (different grids, interfaces and
 * data), Algorithm 1 for each.  The right-hand sides of Step 1 and the final
 * evaluations run as one batched box solve over all instances; the GMRES
 * cycle of all instances is one launch of a captured CUDA graph: a
 * conditional loop whose body is one iteration of every instance (correction
 * values, RHS corrections, box solves and traces each one launch over all
 * instances' work items, then the Arnoldi steps), ended on the device when
 * every instance has converged or the iteration limit is reached.  The batch
 * keeps pointers to the problems, which must outlive it and must not be used
 * for other work while a batched call runs (their operator buffers and
 * box-solver scratch are shared).
 * Requirements: at least one problem; all of one kind (Dirichlet or mu-form
 * interface), with one interface each, on one stream, of one dimension, with box_solver KFBI_BOX_DST,
 * precision KFBI_MIXED, the same Krylov dimension, and N_b <= 32768 each;
 * otherwise KFBI_ERR_UNSUPPORTED (message on problems[0]).  problems: host
 * array of count handles; *out receives the batch (NULL on failure). */
typedef struct kfbi_batch kfbi_batch;
/* Creation also tunes the launch shapes of the batched box solve on the
 * batch's own grids (kfbi_batch_tiles) and synchronises the stream. */
kfbi_status kfbi_create_batch(kfbi_problem* const* problems, int count, kfbi_batch** out);
kfbi_status kfbi_destroy_batch(kfbi_batch* batch);
/* The launch shapes the autotuner picked at kfbi_create_batch: the CTA count
 * of the persistent FP32 transform pass (half, once or twice the CTAs the GPU
 * holds at once) and of the fixed-point row kernel (4, 8, 16 or 32 per SM),
 * each the fastest of its candidates in timed batched box solves with a
 * synthetic right-hand side.  The shapes only distribute work items; results
 * do not depend on them.  Host integers out; KFBI_ERR_ARG on NULL. */
kfbi_status kfbi_batch_tiles(const kfbi_batch* batch, int* pass_ctas, int* row_ctas);
/* Algorithm 1 for every instance k: data[k] (host array of count kfbi_data
 * with device pointers as in kfbi_gmres_solve), x0s (host array of count
 * device pointers, N_b of instance k each, or NULL entries / x0s NULL for a
 * zero start: a start whose residual is not below ||b_k|| (or not finite)
 * is dropped for the zero start, as in kfbi_gmres_solve, infos[k].x0_rejected),
 * densities[k] (host array of count device pointers, N_b each, written),
 * infos (host array of count, may be NULL; t_ms zeroed).  opts applies to
 * every instance; opts->x0 must be NULL; there is no restart: an instance not
 * converged within min(max_iter, restart, Krylov dimension) iterations makes
 * the call return KFBI_ERR_NOT_CONVERGED after writing every density; NaN or
 * Inf data: KFBI_ERR_NONFINITE.  Synchronises the stream three times per call
 * (after the starts, after the GMRES cycle, at the end). */
kfbi_status kfbi_gmres_solve_batch(kfbi_batch* batch, const kfbi_data* data,
                                   const kfbi_gmres_opts* opts, const double* const* x0s,
                                   double* const* densities, kfbi_gmres_info* infos);
/* kfbi_evaluate for every instance from its density, the box solves of all
 * instances as one batched solve: u_grids[k] (host array of count device
 * pointers, (N+1)^d of instance k each) receives instance k's grid solution;
 * data and densities as in kfbi_gmres_solve_batch.  Enqueued on the batch's
 * stream; no synchronisation. */
kfbi_status kfbi_evaluate_batch(kfbi_batch* batch, const kfbi_data* data,
                                const double* const* densities, double* const* u_grids);

/* ---- learned initial density for GMRES ---------------------------------- */

/* A small fully connected network (grown form: learned warm start) maps
 * features of each DOF to an initial density for kfbi_gmres_solve (opts->x0),
 * which falls back to a zero start whenever that guess is not better than zero:
 *   z1 = W1 x~ + b1, a1 = tanh z1;  z2 = W2 a1 + b2, a2 = tanh z2;
 *   y = W3 a2 + b3 + WL x~;  x~ = (x - in_shift) * in_scale;
 *   density = y * out_scale + out_shift  (x: the features of
 *   kfbi_warm_start_features).
 * Parameters are one FP32 vector [W1 (width x n_in, row-major), b1, W2 (width x
 * width), b2, W3 (1 x width), b3, WL (n_in)] owned by the network; the
 * products with W1, W2, W3 use those weights rounded to bfloat16 (round to
 * nearest even); WL, activations and sums are FP32; gradients are those at the
 * rounded weights.  Training uses
 * kfbi_mlp_loss_grad (loss 1/(2n) sum (y - t)^2) and kfbi_mlp_adam (Adam with
 * bias-corrected moments).  All arrays are device arrays unless stated; work
 * is enqueued on the stream given at create. */
#define KFBI_WS_FEATURES 16   /* per-DOF features of kfbi_warm_start_features */
typedef struct kfbi_mlp kfbi_mlp;
/* n_in in [1, 16], width in [1, 1024]; parameters start at zero. */
kfbi_status kfbi_mlp_create(int n_in, int width, void* cuda_stream, kfbi_mlp** out);
kfbi_status kfbi_mlp_destroy(kfbi_mlp* m);
const char* kfbi_mlp_last_error(const kfbi_mlp* m);
kfbi_status kfbi_mlp_num_params(const kfbi_mlp* m, int* count);
/* Copy in the FP32 parameters (count floats) and reset the Adam state. */
kfbi_status kfbi_mlp_set_params(kfbi_mlp* m, const float* params);
/* Copy out the parameters and/or the last gradient (either may be NULL). */
kfbi_status kfbi_mlp_get_params(const kfbi_mlp* m, float* params, float* grads);
/* Input normalisation (HOST arrays of n_in floats) and output affine map. */
kfbi_status kfbi_mlp_set_affine(kfbi_mlp* m, const float* in_shift, const float* in_scale,
                                double out_shift, double out_scale);
/* y (n floats) = network output (before the output affine map) for the rows
 * of X (n x n_in floats, row-major). */
kfbi_status kfbi_mlp_forward(kfbi_mlp* m, const float* X, int n, float* y);
/* Loss and gradient over n rows of X against targets t (in the network's
 * output units): row i of the batch is row rows[i] of X and t (int32 device
 * indices, a minibatch of a shuffled data set), or row i when rows is NULL.
 * loss: one device float (may be NULL). */
kfbi_status kfbi_mlp_loss_grad(kfbi_mlp* m, const float* X, const float* t, const int32_t* rows,
                               int n, float* loss);
/* Parameter groups that kfbi_mlp_adam updates: bit 0 the nonlinear branch
 * (W1, b1, W2, b2, W3), bit 1 the linear part (b3, WL); 3 = all (the
 * default).  Resets the Adam moments and step counter. */
kfbi_status kfbi_mlp_set_trainable(kfbi_mlp* m, int groups);
/* One Adam step with the last gradient (step counter kept by the network). */
kfbi_status kfbi_mlp_adam(kfbi_mlp* m, float lr, float beta1, float beta2, float eps);
/* Per-DOF features (N_b x KFBI_WS_FEATURES floats): [g1, g2, n (3), x (3),
 * level-set parameters p0..p5, log10(sigma_in/sigma_out) (interface kinds;
 * 0 otherwise), 0].  The data are not rescaled per problem (the network's
 * input normalisation, set from its training set, does that per feature).
 * Components beyond the dimension are 0; g2 NULL gives 0.  With density (N_b doubles,
 * e.g. a solved density) also writes target (N_b floats) = the density (FP32):
 * one training sample per DOF.  density and target are both NULL or both given. */
kfbi_status kfbi_warm_start_features(kfbi_problem* p, const kfbi_data* data, const double* density,
                                     float* features, float* target);
/* x0 (N_b doubles) = the network's density for this problem and data.  The
 * network must take KFBI_WS_FEATURES inputs, have width >= KFBI_WS_FEATURES
 * and share the problem's stream. */
kfbi_status kfbi_warm_start(kfbi_problem* p, kfbi_mlp* m, const kfbi_data* data, double* x0);
/* kfbi_warm_start for every instance of a batch with one forward pass of the
 * network over the DOFs of all instances: data (host array of the batch's
 * count kfbi_data) and x0s (host array of count device pointers, N_b of
 * instance k each, written) as in kfbi_gmres_solve_batch.  The network must
 * share the batch's stream. */
kfbi_status kfbi_warm_start_batch(kfbi_batch* batch, kfbi_mlp* m, const kfbi_data* data, double* const* x0s);

/* ---- box solve without allocation ----------------------------------------- */

/* The FP64 sine-transform box solve u = A_h^{-1} rhs of kfbi_box_solve, for a
 * caller that cannot allocate device memory: code whose allocator belongs to
 * someone else (a host application's pool, a plugin or driver layer) or
 * where a cudaMalloc could synchronise the device or fail in the middle of a
 * pipeline.  It needs no kfbi_problem and calls no cudaMalloc, cudaFree or
 * allocating library routine: its scratch (work grid, spectral scale table,
 * twiddles) is one fixed file-scope device array of about 4.4 MB that every GPU
 * loading the library holds until the process exits.  The paper has no
 * counterpart; it is an interface convenience.
 *   dim, n, lo, hi, order, kappa: the grid and the compact operator of
 *     kfbi_config (kappa is kappa~ of the unit-sigma operator Lap - kappa~);
 *   rhs: (N+1)^d device grid, interior nodes read; u: (N+1)^d device grid,
 *     written (boundary layer 0).  Both owned by the caller; they must not
 *     overlap (u is cleared before rhs is read): overlapping ranges return
 *     KFBI_ERR_ARG.
 * Limits: 2D N <= 512, 3D N <= 64 (N a power of two >= 8); larger sizes or
 * invalid arguments return KFBI_ERR_ARG, CUDA failures KFBI_ERR_CUDA.
 * The first call on a device does a one-time set-up (looks up the array's
 * device address and raises shared-memory limits); make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents: calls that overlap on the GPU (different streams, or
 * different host threads) race and give wrong results.  Work is enqueued on
 * cuda_stream. */
kfbi_status kfbi_box_solve_noalloc(int dim, int n, double lo, double hi, int order, double kappa,
                                   const double* rhs, double* u, void* cuda_stream);

/* ---- accounting -------------------------------------------------------- */

/* Kernel launches per class since creation or the last reset (host output of
 * KFBI_KC_COUNT int64 values); reset != 0 zeroes the counters afterwards. */
kfbi_status kfbi_launch_counts(kfbi_problem* p, int64_t* counts, int reset);
/* Enable (1) or disable (0) per-launch timing with CUDA events on the problem's
 * stream; enabling discards earlier records.  Adds host work per launch: keep
 * it off in timed runs. */
kfbi_status kfbi_profile_enable(kfbi_problem* p, int enable);
/* Synchronises the stream and returns, per class, the summed device time (ms)
 * and the number of timed launches since profiling was enabled (host outputs
 * of KFBI_KC_COUNT values each). */
kfbi_status kfbi_profile_read(kfbi_problem* p, double* ms, int64_t* timed_launches);

#ifdef __cplusplus
}
#endif
#endif /* KFBI_H */
