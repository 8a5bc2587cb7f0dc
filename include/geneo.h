/*
 * geneo.h -- C ABI of a GB300 (sm_103a) solver for 3D anisotropic linear
 * elasticity in layered composites: trilinear hexahedral finite elements,
 * preconditioned conjugate gradients with the two-level overlapping additive
 * Schwarz preconditioner and the GenEO coarse space of
 *   Butler, Dodwell, Reinarz, Sandhu, Scheichl, Seelinger, "High-performance
 *   dune modules for solving large-scale, strongly anisotropic elliptic
 *   problems with applications to aerospace composites", arXiv:1901.05188.
 *
 * Conventions (all calls):
 *  - Units are the caller's; the synthetic workloads use mm, N, MPa.
 *  - Mesh: tensor-product nodes x[0..nx], y[0..ny], z[0..nz] (strictly
 *    increasing).  Node n = i + (nx+1)*(j + (ny+1)*k); dof = 3*n + c with
 *    c = 0, 1, 2 for the x, y, z displacement.  Element e = ex + nx*(ey + ny*ez).
 *  - Every array argument may be host memory or device memory of the current
 *    CUDA device; the library finds out with cudaPointerGetAttributes.  Input
 *    arrays stay owned by the caller and are only read during the call.
 *  - All work is ordered on the context's CUDA stream.  Functions returning
 *    data to host memory synchronise that stream before returning.
 *  - Every function returns an int status (GENEO_OK = 0); nothing throws
 *    across the ABI.  geneo_status_string() names a status.
 *  - A context is not thread-safe; use one context per host thread/stream.
 *  - Environment variables, read at geneo_setup (and geneo_batch_create for the
 *    Schwarz pins), fix choices the set-up otherwise makes itself; a value
 *    outside the listed set is ignored:
 *      GENEO_SCHWARZ_CLUSTER  CTAs per subdomain of the local solves: 1, 2, 4, 8
 *      GENEO_SCHWARZ_ROWS     tile rows per step: 1, 2, 4, or 0 (look-ahead)
 *      GENEO_SCHWARZ_STAGED   0 tiles from global memory, 1 staged by bulk
 *                             copies, 2 ring form (local vector streamed)
 *      GENEO_BAND_SOLVE_RING  1: the eigensolver's band solves use the ring form
 *      GENEO_LANCZOS_STEPS    block-Lanczos steps per restart: 10, 12, 16
 *      GENEO_EIG_TOL          Ritz residual bound / theta: 1e-12 .. 1e-4
 *      GENEO_TENSOR_CORES     0: FP32 factor updates on the FMA units
 *    A fixed launch shape gives bit-reproducible results.  Unpinned, the
 *    set-up times the shapes and keeps the fastest (cached per process); two
 *    processes may pick different shapes when they time alike, and different
 *    shapes sum partial products in different orders.
 */
#ifndef GENEO_H
#define GENEO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GENEO_OK = 0,
  GENEO_ERR_INVALID_ARG = 1,
  GENEO_ERR_WORKSPACE_TOO_SMALL = 2,
  GENEO_ERR_CUDA = 3,
  GENEO_ERR_NOT_SPD = 4,          /* non-positive pivot; see stats.failed_subdomain */
  GENEO_ERR_EIG_NOT_CONVERGED = 5,
  GENEO_ERR_CG_BREAKDOWN = 6,     /* p^T A p <= 0 or a NaN in the iteration */
  GENEO_ERR_NOT_CONVERGED = 7,    /* max_it reached; u is still written */
  GENEO_ERR_TIMEOUT = 8,
  GENEO_ERR_UNIMPLEMENTED = 9,
  GENEO_ERR_STATE = 10            /* call order violated (e.g. solve before setup) */
};

typedef struct geneo_ctx geneo_ctx;

/* Precision of the subdomain factors and solves (the bulk of flops and bytes).
 * GENEO_FP64: everything in double; plain PCG.
 * GENEO_MIXED_FP32: subdomain Cholesky factors and triangular solves in single
 *   precision inside an outer double-precision flexible CG; the GenEO
 *   eigensolves, the coarse factor and solve, the residual SpMV and the CG
 *   dot products stay in double. */
typedef enum { GENEO_FP64 = 0, GENEO_MIXED_FP32 = 1 } geneo_precision;

/* One-level term weight D_j in  M^-1 = sum_j R_j^T D_j A_j^-1 R_j + Z A_H^-1 Z^T.
 * GENEO_AS: D_j = I, the symmetric operator of Sec. 3.1 (eqn:onelevelAS).
 * GENEO_AS_POU: D_j = X_j (partition of unity); not symmetric, so solve()
 *   then always uses flexible CG.
 * GENEO_NO_PRECOND: M = I, plain CG (Sec. 3.1 with no preconditioner; the
 *   unpreconditioned baseline the preconditioners are compared with).  The
 *   partition, modes, precision and coarse arguments are then ignored. */
typedef enum { GENEO_AS = 0, GENEO_AS_POU = 1, GENEO_NO_PRECOND = 2 } geneo_schwarz;

/* Coarse space kind. GENEO_COARSE_GENEO: GenEO eigenvectors (Sec. 3.2);
 * GENEO_COARSE_NONE: one-level additive Schwarz only (Sec. 3.1);
 * GENEO_COARSE_ZEM: zero energy modes, the comparison of Sec. 5 (Table 1):
 * the six rigid displacements of every floating subdomain (none for a
 * subdomain touching the Dirichlet boundary), weighted by the same partition
 * of unity; the mode options other than the shift are ignored. */
typedef enum { GENEO_COARSE_GENEO = 0, GENEO_COARSE_NONE = 1, GENEO_COARSE_ZEM = 2 } geneo_coarse;

/* Partition of unity X_j (Def. Partition of Unity, Sec. 3.2; Sec. 3.3.1),
 * used in B_j = X_j A_{Omega_j^o} X_j, in the coarse basis R_j^T X_j p and in
 * the one-level weight D_j = X_j of GENEO_AS_POU.
 * GENEO_POU_MULTIPLICITY: 1 / (number of subdomains whose V_{h,0} holds the
 *   node), Sec. 3.3.1 (the default).
 * GENEO_POU_SARKIS: d_j / sum_k d_k, d_j the node's distance to the
 *   artificial boundary of Omega_j counted in element layers (the least
 *   distance to a face of Omega_j's box that lies inside the domain; 1 when
 *   there is none), the sum over the subdomains whose V_{h,0} holds the
 *   node: Sarkis's smoother partition of unity, Sec. 3.2.  Equal to the
 *   multiplicity one at overlap 1.
 * Both are zero on global Dirichlet dofs and on Omega_j's artificial
 * boundary. */
typedef enum { GENEO_POU_MULTIPLICITY = 0, GENEO_POU_SARKIS = 1 } geneo_pou;

/* Solver of the coarse problem A_H y = w (Sec. 3.3.3).
 * GENEO_COARSE_DIRECT: Cholesky factor of A_H at set-up, its explicit inverse
 *   applied as a matrix-vector product (the default).
 * GENEO_COARSE_ITERATIVE: the inexact solve the paper uses for very large
 *   coarse spaces: CG on A_H from y = 0, preconditioned by the inverses of
 *   A_H's diagonal blocks (one block per subdomain's modes), stopped at
 *   ||w - A_H y|| <= tol ||w|| or after max_it steps; the outer Krylov method
 *   is then flexible CG.  The paper preconditions this inner CG with an
 *   algebraic multigrid (BoomerAMG); block Jacobi stands in for it here. */
typedef enum { GENEO_COARSE_DIRECT = 0, GENEO_COARSE_ITERATIVE = 1 } geneo_coarse_solver;

typedef struct {
  int nx, ny, nz;                 /* elements per axis, each >= 1 */
  const double *x, *y, *z;        /* node coordinates, lengths nx+1, ny+1, nz+1 */
} geneo_mesh;

/* Orthotropic material in its own axes (Sec. 2: nine constants; isotropic
 * resin as E1=E2=E3=E, G=E/(2(1+nu)), nu12=nu13=nu23=nu). */
typedef struct {
  double E1, E2, E3, G12, G13, G23, nu12, nu13, nu23;
} geneo_ortho;

typedef struct {
  int n;                          /* number of constrained dofs */
  const int32_t *dof;             /* constrained dofs, 3*node + c, each < 3*nodes */
  const double *value;            /* prescribed displacement per entry */
} geneo_dirichlet;

/* Box partition: the elements of each axis split into p parts
 * [floor(k n / p), floor((k+1) n / p)), each grown by `overlap` element
 * layers (Sec. 3.1).  Subdomain j = jx + px*(jy + py*jz). */
typedef struct {
  int px, py, pz;
  int overlap;                    /* >= 1 */
} geneo_partition;

/* GenEO mode selection (Sec. 3.2): fixed_modes > 0 keeps exactly that many
 * eigenvectors per subdomain; otherwise all with lambda <= threshold, where
 * threshold <= 0 selects diam(Omega_j)/width(Omega_j^o) (box circumradius over
 * O times the smallest element edge), capped at max_modes.  A cut inside a
 * cluster of equal eigenvalues (relative gap <= 1e-6) drops the cluster.
 * shift < 0 is the shift-and-invert shift sigma (Sec. 3.3.2). */
typedef struct {
  int fixed_modes;
  double threshold;
  int max_modes;                  /* 1..32 */
  double shift;
} geneo_modes;

typedef struct {
  int iterations;                 /* A p products performed by (F)PCG */
  double rel_res_recursive;       /* ||r_k|| / ||b|| of the recursion at exit */
  double rel_res_true;            /* ||b - A u|| / ||b|| recomputed at exit */
  double kappa_est;               /* Lanczos estimate from the CG coefficients (PCG only, else 0) */
  int n_coarse;                   /* N_H = sum_j m_j */
  int n_subdomains;
  /* CUDA-event times; the subdomain factorisation (ms_setup_factor) runs on its
   * own streams concurrently with the GenEO eigensolve (ms_setup_eig) */
  float ms_assemble, ms_setup_eig, ms_setup_coarse, ms_setup_factor, ms_solve;
  double bytes_per_iter;          /* algorithmic HBM bytes of one iteration */
  double eig_max_residual;        /* max Ritz residual of the kept eigenpairs */
  int failed_subdomain;           /* subdomain of a GENEO_ERR_NOT_SPD, else -1 */
  int flexible;                   /* 1 if flexible CG was used */
  int eig_cycles;                 /* block-Lanczos restart cycles of the last set-up */
  int lanczos_steps;              /* block-Lanczos steps of the last set-up (two band sweeps each) */
  int schwarz_cluster;            /* CTAs per subdomain chosen for the local solves */
  int schwarz_rows;               /* tile rows per cluster barrier chosen for them */
  int schwarz_staged;             /* 1 if their tiles are staged in shared memory by bulk copies,
                                     2 if the local vector streams through a ring of tile rows
                                     (subdomains whose local vector exceeds shared memory) */
  int coarse_inner_iterations;    /* inner PCG steps of the iterative coarse solve, summed over
                                     the solve's preconditioner applications (0 if direct) */
} geneo_stats;

/* Create a context whose work runs on `cuda_stream` (a cudaStream_t; NULL =
 * legacy default stream) on the current CUDA device. */
int geneo_create(geneo_ctx **out, void *cuda_stream);
int geneo_destroy(geneo_ctx *ctx);
const char *geneo_status_string(int status);
/* Human-readable detail of the last failure on this host thread. */
const char *geneo_last_error(void);
/* Number of kernel launches this library has enqueued in this process so far
 * (a CUDA-graph launch counts its kernel nodes).  Not thread-safe. */
long long geneo_launch_count(void);

/* Device bytes needed by geneo_assemble for this mesh (BSR matrix, load,
 * per-element material data, index arrays). */
int geneo_assemble_workspace_bytes(const geneo_mesh *mesh, size_t *bytes);

/* Device bytes needed by geneo_setup + geneo_solve for this partition, mode
 * cap and precision (subdomain factors, eigensolver, coarse space, Krylov
 * vectors).  Call after geneo_assemble. */
int geneo_setup_workspace_bytes(geneo_ctx *ctx, const geneo_partition *part,
                                const geneo_modes *modes, geneo_precision prec,
                                size_t *bytes);

/* Host-only estimate of both workspaces (assemble, setup + solve) for a
 * problem that has not been assembled yet; used to admit requests by device
 * memory.  unknowns_per_node: 3 for elasticity (geneo_assemble), 1 for the
 * Darcy problem (geneo_assemble_darcy); the assemble figure is the
 * elasticity one, an upper bound for Darcy.  Either output may be NULL.
 * Touches no device state. */
int geneo_estimate_workspace_bytes(const geneo_mesh *mesh, int unknowns_per_node,
                                   const geneo_partition *part, const geneo_modes *modes,
                                   geneo_precision prec, size_t *assemble_bytes,
                                   size_t *setup_bytes);

/* Host-only view of the subdomain plan geneo_setup builds for this mesh and
 * box partition (Sec. 3.1: parts of each axis with n elements and p parts
 * own [floor(k n / p), floor((k + 1) n / p)); Omega_j adds `overlap` element
 * layers per side, clipped to the mesh; V_{h,0}(Omega_j) keeps the nodes of
 * Omega_j not on its boundary inside the domain).  Subdomain j = kx + px (ky
 * + py kz) fills GENEO_PLAN_INTS int32 at plan[GENEO_PLAN_INTS * j]: element
 * box lo (x, y, z) and hi (exclusive), interior node box lo and hi (inclusive),
 * then the interior unknown count n_j and the half-bandwidth of its band
 * factor in 32-row tiles, and the same two for the Neumann set (all nodes of
 * Omega_j).  *n_subdomains = px py pz; with plan NULL only the count is
 * returned; max_subs below the count is GENEO_ERR_INVALID_ARG.  The
 * partition is refused (GENEO_ERR_INVALID_ARG) exactly when geneo_setup
 * would refuse it: parts outside [1, elements] on an axis, an empty interior,
 * or an overlap so wide that a node lies in the interiors of more than four
 * parts of one axis (the gather's candidate lists hold four).  Touches no
 * device state. */
#define GENEO_PLAN_INTS 16
int geneo_plan_subdomains(const geneo_mesh *mesh, int unknowns_per_node,
                          const geneo_partition *part, int max_subs, int32_t *plan,
                          int *n_subdomains);

/* Bind caller-owned device memory (e.g. allocated by PyTorch) as the
 * workspace of phase 0 (assemble) or phase 1 (setup + solve).  It must stay
 * alive until the context is destroyed or rebound; alignment >= 256 bytes.
 * A phase run without a bound workspace allocates its own with cudaMalloc
 * (freed by geneo_destroy).  Too small a workspace makes the phase return
 * GENEO_ERR_WORKSPACE_TOO_SMALL. */
int geneo_bind_workspace(geneo_ctx *ctx, int phase, void *device_ptr, size_t bytes);

/* Assemble A u = b (Sec. 2, eqn:fe_matrix_system) on the device:
 * per-element orthotropic stiffness rotated by the ply angle theta about +z
 * and the out-of-plane angle phi (fibre direction
 * (cos t cos p, sin t cos p, -sin p)); Q1 element stiffness by 2x2x2 Gauss
 * integration; 3x3-block BSR; symmetric elimination of the Dirichlet dofs
 * (b -= A[:,D] g, rows/cols zeroed, unit diagonal, b_D = g); load = consistent
 * nodal forces of the traction (0, 0, -top_pressure) on the face z = z_max
 * plus `nodal_load` (length 3*nodes, may be NULL).
 *   elem_mat  : int32[nel], material index < n_mat
 *   elem_theta: double[nel], radians
 *   elem_phi  : double[nel], radians, may be NULL (all zero) */
int geneo_assemble(geneo_ctx *ctx, const geneo_mesh *mesh, int n_mat,
                   const geneo_ortho *mats, const int32_t *elem_mat,
                   const double *elem_theta, const double *elem_phi,
                   const geneo_dirichlet *dirichlet, const double *nodal_load,
                   double top_pressure);

/* Assemble the scalar Darcy problem of the paper's subsurface application
 * (the section on the SPE10 benchmark, eqn:Darcy and eq-fe-darcy):
 * -div(K grad u) = f with K = diag(Kx, Ky, Kz) constant per element, Q1
 * elements with 2x2x2 Gauss integration, one unknown per node (dof = node),
 * 1x1 blocks in the same 27-point BSR pattern, symmetric elimination of the
 * Dirichlet set.  Everything after it -- geneo_setup (GenEO, ZEM or none,
 * FP64 or mixed), geneo_solve, geneo_set_load (its scalar is the source f) --
 * works on this system as on the elasticity one; geneo_element_stress does not.
 *   perm      : 3*n_elements doubles (Kx, Ky, Kz) per element (host or device)
 *   dirichlet : node ids and values (e.g. the face z = 0 with u = 0)
 *   nodal_load: n_nodes doubles added to the right-hand side, may be NULL
 *   source    : uniform f, applied as int f N_a dx */
int geneo_assemble_darcy(geneo_ctx *ctx, const geneo_mesh *mesh, const double *perm,
                         const geneo_dirichlet *dirichlet, const double *nodal_load,
                         double source);

/* Replace the load of the assembled system (Sec. 2, the right-hand side of
 * eqn:fe_matrix_system) without touching the matrix, the preconditioner or
 * the captured iteration: b = f + lift on free rows and b_D = g, where f is
 * the traction (0, 0, -top_pressure) on z = z_max plus `nodal_load` (host or
 * device, 3*nodes doubles, may be NULL) and lift = -A[:,D] g is kept from
 * geneo_assemble (same Dirichlet set and values).  The next geneo_solve
 * solves with the new b.  Errors: GENEO_ERR_STATE before geneo_assemble. */
int geneo_set_load(geneo_ctx *ctx, const double *nodal_load, double top_pressure);

/* Stress recovery (Sec. 2 constitutive law; the stresses the paper derives
 * from the displacements for its failure analysis, Sec. 5): for every element
 * sigma = C_e B(centre) u_e, the rotated ply stiffness times the strain of the
 * trilinear element at its centre (its element-average strain).
 *   u     : 3*n_nodes doubles (host or device), e.g. from geneo_solve
 *   sigma : 6*n_elements doubles (host or device), element e at 6e, Voigt
 *           order (xx, yy, zz, yz, xz, xy), element e = ex + nx*(ey + ny*ez)
 * Errors: GENEO_ERR_STATE before geneo_assemble. */
int geneo_element_stress(geneo_ctx *ctx, const double *u, double *sigma);

/* Sizes of the assembled system: nodes and stored 3x3 blocks. */
int geneo_system_info(geneo_ctx *ctx, int *n_nodes, int *nnz_blocks);

/* Copy the assembled BSR (row_ptr[n_nodes+1], col[nnzb], val[9*nnzb] with
 * each block row-major) and the load b[3*n_nodes]; any pointer may be NULL. */
int geneo_get_system(geneo_ctx *ctx, int32_t *row_ptr, int32_t *col,
                     double *val, double *b);

/* y = A x with the assembled matrix (x, y: 3*n_nodes doubles). */
int geneo_spmv(geneo_ctx *ctx, const double *x, double *y);

/* Build the preconditioner (Sec. 3.1-3.3): subdomains, partition of unity,
 * GenEO eigenproblems A_{Omega_j} p = lambda X_j A_{Omega_j^o} X_j p by
 * shift-and-invert block Lanczos, coarse basis Z = [R_j^T X_j p_k], coarse
 * matrix A_H = Z^T A Z and its Cholesky factor, and the band Cholesky factors
 * of A_j = R_j A R_j^T in the requested precision.  Subdomain size is bounded
 * by device memory only: a local vector too large for shared memory is
 * streamed through it (GENEO_ERR_INVALID_ARG only for a half-bandwidth above
 * about 27,000 unknowns, the ring of tile rows the FP64 sweeps keep). */
int geneo_setup(geneo_ctx *ctx, const geneo_partition *part,
                const geneo_modes *modes, geneo_precision prec,
                geneo_schwarz schwarz, geneo_coarse coarse);

/* Partition of unity of the next geneo_setup calls on this context
 * (geneo_pou; the default is GENEO_POU_MULTIPLICITY).  Host-only; returns
 * GENEO_ERR_INVALID_ARG for an unknown kind. */
int geneo_set_partition_of_unity(geneo_ctx *ctx, int kind);

/* Coarse solver of the next geneo_setup calls on this context
 * (geneo_coarse_solver; tol and max_it are read for GENEO_COARSE_ITERATIVE
 * only: 0 < tol < 1, max_it >= 1).  Host-only; GENEO_ERR_INVALID_ARG
 * otherwise.  The iterative solve runs as one cooperative launch per
 * application: its blocks wait for one another at a grid barrier (bounded:
 * after about a second the solve fails with GENEO_ERR_TIMEOUT). */
int geneo_set_coarse_solver(geneo_ctx *ctx, int kind, double tol, int max_it);

/* z = M^-1 r with the preconditioner of the last geneo_setup. */
int geneo_apply_preconditioner(geneo_ctx *ctx, const double *r, double *z);

/* Coarse-space summary: per subdomain the kept mode count m_j
 * (modes[n_subdomains]) and the smallest (max_modes+1) eigenvalues
 * (lambdas[n_subdomains*(max_modes+1)], +inf where not computed/infinite).
 * Any pointer may be NULL. */
int geneo_coarse_info(geneo_ctx *ctx, int *n_subdomains, int *n_coarse,
                      int32_t *modes, double *lambdas);

/* Dense copies for inspection: Phi[3*n_nodes x n_coarse] column-major coarse
 * basis; AH[n_coarse x n_coarse] coarse matrix.  Either may be NULL. */
int geneo_get_coarse(geneo_ctx *ctx, double *Phi, double *AH);

/* Inspection of one subdomain's matrices, assembled afresh on the device:
 * kind 0: A_j = R_j A R_j^T on the dofs of V_{h,0}(Omega_j) (Sec. 3.1);
 * kind 1: S_j = A_{Omega_j} - shift * X_j A_{Omega_j^o} X_j on all dofs of
 *         Omega_j (the shifted GenEO pencil, Sec. 3.3.2);
 * kind 2: B_j = X_j A_{Omega_j^o} X_j (eqm:matrixForm);
 * kind 3, 4: the band Cholesky factor of kind 0, 1 computed afresh in FP64:
 *         the dense lower block-band with each 32 x 32 diagonal block
 *         replaced by its inverse (the storage the triangular sweeps use).
 * dense: n x n row-major (n = 3 x nodes of the set; NULL to skip); gdof[n]:
 * global dof of each local row (may be NULL).  Needs a preceding geneo_setup
 * call (it may have failed after planning); kinds 1, 2, 4 need the GenEO
 * coarse space.  Allocates scratch with cudaMallocAsync. */
int geneo_debug_local_matrix(geneo_ctx *ctx, int sub, int kind, double *dense, int32_t *gdof);

/* Time `reps` back-to-back launches of one hot kernel on the context stream
 * with CUDA events (after one warm-up launch) and report its algorithmic
 * traffic: what 0 = the one-level Schwarz local solves (Sec. 3.1,
 * eqn:onelevelAS: gather, forward and backward band sweeps, both factor
 * streams), 1 = the BSR SpMV, 2 = the whole preconditioner application,
 * 3 = one FP64 backward sweep of the GenEO eigensolver's band solves with 8
 * right-hand sides per subdomain (Sec. 3.3.2 shift-and-invert operator),
 * 4 = the band Cholesky factorisation of the shifted Neumann matrices
 * S_j = A_Omega_j - sigma B_j (FP64, re-assembled first; Sec. 3.3.2),
 * 5 = the band Cholesky factorisation of the subdomain matrices A_j in the
 * set-up's precision (re-extracted first; Sec. 3.1 local solves).  Kinds 4
 * and 5 rebuild the factors they time, with the same result.
 * Outputs (any may be NULL): mean ms per launch, bytes and flops per launch.
 * Needs geneo_setup; overwrites the solver's internal work vectors. */
int geneo_profile(geneo_ctx *ctx, int what, int reps, double *ms_per_launch, double *bytes,
                  double *flops);

/* y = A x and *xy = x . y for a 3x3-block BSR matrix, without allocating.
 * This entry point has no counterpart in the paper: it serves callers that
 * cannot allocate device memory (a host framework that hands out a fixed
 * device-memory budget, a real-time loop that must not enter the CUDA
 * allocator, a plug-in that only receives pointers to someone else's
 * buffers).  It calls no cudaMalloc, cudaFree or allocating library routine.
 * Its only scratch is a file-scope device array of 65,536 partial sums
 * (512 KiB, held by every GPU that loads the library until exit), so n_nodes
 * may be at most 524,288 block rows; larger inputs return
 * GENEO_ERR_WORKSPACE_TOO_SMALL.  All pointers are device memory owned by the
 * caller: row_ptr[n_nodes+1], col[nnzb], val[9*nnzb] (row-major blocks;
 * rows may hold any number of blocks), x and y [3*n_nodes], xy [1].  x and y
 * must not overlap (GENEO_ERR_INVALID_ARG otherwise).  Work is enqueued on cuda_stream (NULL = legacy
 * default stream); the call does not synchronise.  The first call on each
 * device looks up the scratch array's device address (cudaGetSymbolAddress)
 * with that device current, so make that first call before any stream
 * capture.  Every call shares the scratch and clears its counter on entry:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. */
int geneo_spmv_dot_noalloc(int n_nodes, const int32_t *row_ptr, const int32_t *col,
                           const double *val, const double *x, double *y, double *xy,
                           void *cuda_stream);

/* The set-up's mode-selection rule (Sec. 3.2), host-only: given n eigenvalues
 * in ascending order (INFINITY for infinite ones), *m = modes->fixed_modes
 * when that is > 0 (at most the finite ones), else the number of eigenvalues
 * <= tau capped at modes->max_modes; then, while the cut falls inside a
 * cluster (neighbours equal to 1e-6 relative plus 1e-9), one fewer, so the
 * kept span is unique. */
int geneo_select_modes(const double *lambdas, int n, const geneo_modes *modes, double tau,
                       int *m);

/* The set-up's default eigenvalue thresholds (Sec. 3.2 and its footnote, read
 * for a 3D box): per subdomain, half the diagonal of Omega_j's box over
 * overlap times its smallest element edge.  The mesh coordinates are host
 * arrays here.  *n_subdomains as for geneo_plan_subdomains; tau may be NULL.
 * Host-only. */
int geneo_default_thresholds(const geneo_mesh *mesh, const geneo_partition *part, int max_subs,
                             double *tau, int *n_subdomains);

/* The condition estimate geneo_solve reports (stats.kappa_est), from the CG
 * coefficients alpha_0..alpha_{k-1} and beta_0..beta_{k-2} of a plain PCG run
 * (host arrays): the ratio of the extreme eigenvalues of the Lanczos
 * tridiagonal T with T_ii = 1/alpha_i + beta_{i-1}/alpha_{i-1} and
 * T_{i,i+1} = sqrt(beta_i)/alpha_i (the estimate of Sec. 5, Tables 1-2),
 * found by Sturm-sequence bisection.  0 when k = 0 or the smallest
 * eigenvalue is not positive.  Host-only. */
int geneo_kappa_from_cg(const double *alphas, const double *betas, int k, double *kappa);

/* Batched solves (the many-instance form of geneo_solve, for a stream of
 * independent problems of uneven sizes; Sec. 3.3's batched local solves
 * carried across instances).  A batch is built from n contexts that are each
 * assembled and set up (same device, same precision, the direct coarse
 * solve); it keeps their matrices, factors and coarse spaces where they are
 * and owns only the concatenated Krylov vectors and its work tables.  Every
 * kernel launch of an iteration covers every instance; each instance keeps
 * its own (F)PCG scalars and stops on its own criterion; the one-level local
 * solves of all instances run in one persistent launch whose CTAs take
 * (instance, subdomain) items from a device work queue, largest first, in a
 * launch shape chosen by timing at creation (GENEO_SCHWARZ_ROWS /
 * GENEO_SCHWARZ_STAGED pin it); the iterations are captured in a CUDA graph.
 * While a batch exists its contexts must not run other work (it uses their
 * buffers).  Work goes to cuda_stream (NULL = legacy default stream).
 * Returns GENEO_ERR_STATE for a context that is not set up,
 * GENEO_ERR_INVALID_ARG for mixed precisions or devices, a repeated context,
 * or a subdomain whose local vector does not fit in shared memory (the
 * batched local solves hold it whole). */
typedef struct geneo_batch geneo_batch;
int geneo_batch_create(geneo_batch **out, geneo_ctx *const *ctxs, int n, void *cuda_stream);

/* Solve every instance of the batch from u0 = 0 to ||r_k|| <= tol ||b_k||
 * or max_it iterations (Sec. 3.1), each with its context's current
 * right-hand side (geneo_set_load may change it between solves).  u[i] (host or device, 3*n_nodes or n_nodes
 * doubles; NULL entries skipped) receives instance i's solution; stats[i]
 * (may be NULL) its statistics, ms_solve being the whole batch's time.
 * Returns GENEO_ERR_NOT_CONVERGED / GENEO_ERR_CG_BREAKDOWN if any instance
 * did not converge (the others' results are still written). */
int geneo_batch_solve(geneo_batch *batch, double tol, int max_it, double *const *u,
                      geneo_stats *stats);

int geneo_batch_destroy(geneo_batch *batch);

/* Solve A u = b by PCG (FP64 precision, GENEO_AS) or flexible CG (mixed
 * precision or GENEO_AS_POU) from u0 = 0 until ||r_k|| <= tol ||b|| or max_it
 * iterations (Sec. 3.1).  u: 3*n_nodes doubles.  stats may be NULL. */
int geneo_solve(geneo_ctx *ctx, double tol, int max_it, double *u,
                geneo_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* GENEO_H */
