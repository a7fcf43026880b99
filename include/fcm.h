/*
 * fcm.h - C ABI of the GB300 hierarchical multigrid solver for the finite
 * cell method (Jomo et al., "Hierarchical multigrid approaches for the finite
 * cell method on uniform and multi-level hp-refined grids", arXiv 2010.00881).
 *
 * Problem (Sec. 2.1, Eq. weakform): find u_h with
 *   int (B v)^T alpha C B u dOmega + int beta (N v)^T N u dGamma_D
 *     = int alpha (N v)^T f dOmega + int (N v)^T g_N dGamma_N
 *       + int beta (N v)^T g_D dGamma_D
 * on a uniform Cartesian grid of integrated Legendre elements of degree p
 * (tensor-product space), alpha = 1 in the physical domain {psi <= 0} and
 * alpha = eps << 1 in the fictitious domain.
 *
 * Solver (Sec. 3 and 4): conjugate gradients preconditioned by one
 * hierarchical multigrid V-cycle (Algorithm 1) per iteration: elementwise
 * additive Schwarz smoothing (Eq. AdditiveSchwarz) with n_pre / n_post steps,
 * binary p-transfers (Eq. restrictionoperation) down the arithmetic
 * p-sequence, nested Q1 h-coarsening below p = 1 (the Remark of Sec. 3.2)
 * and a dense Cholesky solve on the coarsest grid.
 *
 * Conventions (all entry points):
 *  - Every vector is a caller-owned buffer of `ndofs` doubles in the
 *    hierarchical layout: per axis the 1D index of node k is k and that of
 *    the degree-q bubble of cell c is (C+1) + (q-2) C + c; the scalar index
 *    is ix + m_x (iy + m_y iz) with m = C p + 1; vector fields (elasticity)
 *    stack whole scalar fields.  `_dev` pointers are device memory of the
 *    device current at setup, `_host` pointers host memory.
 *  - With trunk-space elements (fcm_grid.space) the vectors keep this
 *    layout: inputs' entries on the removed modes are ignored (a solve's
 *    b_dev is taken as zero there) and every output is zero there.
 *  - The handle owns all device state (matrices, inverses, work vectors,
 *    captured graphs) and frees it in fcm_destroy.  All work is ordered on
 *    the CUDA stream given at setup; calls return after that stream has
 *    finished the call's work unless stated otherwise.
 *  - No exception or C++ object crosses the ABI.  On failure the status is
 *    returned and fcm_last_error() describes it (thread-local string, valid
 *    until the next call on the same thread).  A NULL handle or pointer, an
 *    invalid enum or size gives FCM_E_INVALID; CUDA failures FCM_E_CUDA.
 */
#ifndef FCM_H
#define FCM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FCM_OK = 0,
  FCM_E_INVALID = 1,       /* bad argument, NaN input, inconsistent descriptor */
  FCM_E_OOM = 2,           /* device allocation failed */
  FCM_E_CUDA = 3,          /* CUDA runtime error (message in fcm_last_error) */
  FCM_E_UNSUPPORTED = 4,   /* valid request this build does not implement */
  FCM_E_NOT_CONVERGED = 5, /* maxit reached; x holds the last iterate */
  FCM_E_BREAKDOWN = 6,     /* CG breakdown: p^T A p <= 0 or non-finite scalar */
  FCM_E_TIMEOUT = 7        /* a bounded device-side wait expired */
} fcm_status;

/* Arithmetic of the preconditioner (the outer CG is always FP64). */
typedef enum {
  FCM_FP64 = 0,  /* everything in FP64 */
  FCM_MIXED = 1  /* FP32 V-cycle with FP64-accurate islands inside FP64 flexible CG */
} fcm_precision;

enum { FCM_GEOM_NONE = 0, FCM_GEOM_BALL = 1, FCM_GEOM_VOIDS = 2, FCM_GEOM_ELLIPSOID = 3,
       FCM_GEOM_POPCORN = 4 };
enum { FCM_PDE_POISSON = 0, FCM_PDE_ELASTICITY = 1 };
enum { FCM_SRC_CONST = 0, FCM_SRC_SIN3 = 1, FCM_SRC_SQUARE_MMS = 2, FCM_SRC_POPCORN = 3 };
enum { FCM_DIR_NONE = 0, FCM_DIR_LEVELSET = 1, FCM_DIR_FACES = 2 };
enum { FCM_G_ZERO = 0, FCM_G_SIN3 = 1, FCM_G_SQUARE_MMS = 2, FCM_G_POPCORN = 3 };
enum { FCM_SMOOTHER_ELEMENTWISE = 0, FCM_SMOOTHER_PATCHWISE = 1, FCM_SMOOTHER_JACOBI = 2 };

/* Grid: dim in {2,3}; cells per axis (>= 1); box [lo, hi]; degree p in
 * [1, 8].  overlay_levels > 0 (multi-level hp) is FCM_E_UNSUPPORTED in
 * fcm_setup; fcm_mlhp_create builds the overlay topology on the host.
 * space: FCM_SPACE_TENSOR (Q_p on every cell) or FCM_SPACE_TRUNK, the
 * trunk space of Sec. 4.3 (of the tensor modes, those whose bubble degrees
 * sum to at most p; the p-levels use the trunk spaces of their degrees).
 * With trunk elements vectors keep the tensor layout: the other modes are
 * removed from the system (zero rows, columns, loads and corrections) and
 * stay zero in every result; fcm_level_info.ndofs_active counts the rest.
 * drop_outside: 1 removes the cells classified outside the physical domain
 * together with the DOFs supported only on them (Sec. 4.3 and 4.3.2; trunk
 * space only): their matrices, loads and blocks are left out, the Q1
 * h-levels keep the coarse nodes some kept fine node depends on, and the
 * removed DOFs keep their slots in the vectors like removed trunk modes. */
enum { FCM_SPACE_TENSOR = 0, FCM_SPACE_TRUNK = 1 };
typedef struct {
  int dim;
  int cells[3];
  double lo[3], hi[3];
  int p;
  int overlay_levels;
  int overlay_p;
  int space;
  int drop_outside;
} fcm_grid;

/* Level-set geometry, Omega_phys = {psi <= 0}.  params (host memory, read
 * during fcm_setup only):
 *   BALL       cx cy [cz] r                          psi = |x-c| - r
 *   VOIDS      n_params/4 balls (cx cy cz r; cz unused in 2D)   psi = max_k (r_k - |x-c_k|)
 *   ELLIPSOID  cx cy cz a0 a1 a2 R00 R01 ... R22      psi = |diag(1/a) R^T (x-c)| - 1
 *   POPCORN    r0 A sigma, then bump centres (cx cy cz)...  (3D, Sec. 4.3.2)
 *              psi = |x| - r0 - sum_k A exp(-|x - c_k|^2 / sigma^2)
 * Cell and sub-cell classification: exact nearest/farthest distances for
 * balls and voids, a 5^d lattice sign test for the ellipsoid and the
 * popcorn.
 * complement: 0 keeps Omega_phys = {psi <= 0}; 1 makes the other side
 * physical, Omega_phys = {psi >= 0} (a hole instead of an inclusion): psi
 * is negated and the box classification swaps inside and outside (cut
 * stays), so the cut cells and their space trees are the same.  The field
 * is last and zero keeps the usual side, so zero-initialised descriptors
 * are unaffected. */
typedef struct {
  int kind;
  int n_params;
  const double* params;
  int complement;
} fcm_geometry;

/* Physics of Eq. (weakform).  Poisson: kappa scales the stiffness.
 * Elasticity: isotropic E, nu (3D).  alpha: fictitious factor; beta:
 * penalty.  source: CONST (f = f0), SIN3 (f = kappa d pi^2 prod sin(pi x_a)),
 * SQUARE_MMS (f = cos(a x') sin(a y'), x' = x - 1/2, y' = y - 1/2, a = src_a),
 * POPCORN (f = -kappa Lap u for the manufactured u = x^3 + x y^2 + y^3 + z^4
 * + sin(3 (x^2 + y^2)) of Sec. 4.3.2; g POPCORN is that u).
 * dirichlet: LEVELSET (penalty on {psi = 0}) or FACES (bit 2a+s of
 * dirichlet_faces: face of axis a, lower s = 0 / upper s = 1); g selects
 * g_D.  traction_face (-1: none) carries the constant traction vector.
 * quad_depth: space-tree depth on cut cells (0..4).  quadrature: how the
 * cell matrices are summed on each space-tree leaf (the same Gauss points
 * either way, results equal up to rounding): FCM_QUAD_POINTS (0) point by
 * point; FCM_QUAD_SUMFACT (1) by sum factorisation over the leaf's tensor
 * grid of points, one axis at a time (leaves of at most 128 points, i.e.
 * p <= 4 in 3D; others point by point). */
enum { FCM_QUAD_POINTS = 0, FCM_QUAD_SUMFACT = 1 };
typedef struct {
  int pde;
  double kappa, E, nu;
  double alpha, beta;
  int source;
  double f0;
  double src_a;
  int dirichlet;
  int g;
  unsigned dirichlet_faces;
  int traction_face;
  double traction[3];
  int quad_depth;
  int quadrature;
} fcm_physics;

/* Solver options.  smoother: ELEMENTWISE additive Schwarz (Sec. 3.3.1), or
 * JACOBI, the pointwise comparison smoother of Sec. 4.1 (x += omega D^{-1} r,
 * D = diag(A_l); omega <= 0 selects 2/3); PATCHWISE is FCM_E_UNSUPPORTED
 * here (patchwise blocks run through fcm_mlhp_op_prepare, on uniform grids
 * with grid->overlay_levels = 0).
 * For ELEMENTWISE omega <= 0 selects the paper's values (Sec. 3.3.2),
 * clamped per level to 1.75 / lambda_max(M^{-1} A) where that value would
 * break the stability condition rho(I - omega M^{-1} A) < 1.  n_pre, n_post:
 * smoothing steps (paper: 5, 5).  coarse_cells: h-coarsening stops once
 * every axis has at most this many cells (>= 1).  build_mixed: also build
 * the FP32 data of FCM_MIXED. */
typedef struct {
  int smoother;
  double omega;
  int n_pre, n_post;
  int coarse_cells;
  int build_mixed;
} fcm_solver_opts;

typedef struct {
  int iters;                 /* CG iterations (= V-cycles after the first) */
  double relres_recursive;   /* ||r_k|| / ||b|| of the CG recurrence */
  double relres_true;        /* ||b - A x|| / ||b|| recomputed at the end */
  double setup_ms;           /* wall time of fcm_setup */
  double solve_ms;           /* wall time of this solve (host clock) */
  long long ndofs;
  long long kernel_launches; /* device kernels this solve launched (graph nodes included) */
  long long bytes_moved_est; /* algorithmic bytes of this solve: every launch's stored
                                matrices once, its input and output vectors once (the
                                per-kernel byte model of fcm_op_bytes), summed over the
                                launches made; divided by solve_ms, the solve's
                                effective bandwidth */
  double setup_phase_ms[5];  /* fcm_setup by phase, timed by CUDA events on the handle's
                                stream (host work between launches included): [0] geometry
                                (classification, space-tree integration of the cut cells,
                                load), [1] level hierarchy (p-levels, Galerkin h-levels),
                                [2] coarse factorisation, [3] smoothers (block
                                factorisation and inversion, omega estimates), [4] V-cycle
                                graph capture; zero for handles not made by fcm_setup */
} fcm_info;

/* Per-level description (test and benchmark introspection). */
typedef struct {
  int cells[3];
  int p;
  int is_h_level;            /* 1: Q1 Galerkin level below p = 1 */
  long long ndofs;
  int nloc;                  /* DOFs per cell */
  int n_own_cells;           /* cells with a stored matrix (the rest share s K_ref) */
  int n_own_blocks;          /* AS blocks with a stored inverse */
  int n_fp64_blocks;         /* of those, kept in FP64 by FCM_MIXED */
  double omega;              /* relaxation used on this level (0 on level 0) */
  double lambda_est;         /* estimate of lambda_max(M^{-1} A) */
  double max_block_cond;     /* largest infinity-norm condition number of the stored
                                AS blocks, diagonally scaled (0: none stored) */
  int fp64_in_mixed;         /* 1: the FCM_MIXED V-cycle runs this level in FP64 (the
                                finest level when its blocks reach 1e12, or a
                                single-level hierarchy) */
  int kron_operator;         /* 1: the FP64 operator applies its shared (uncut Poisson)
                                cells by sum factorisation of the Kronecker-sum cell
                                matrix instead of the dense matrix */
  long long ndofs_active;    /* DOFs of the level's space (ndofs unless trunk) */
} fcm_level_info;

typedef struct fcm_handle fcm_handle;

/* Discretise, assemble on the device, build the multigrid hierarchy (level
 * matrices, AS inverses, Galerkin h-levels, coarse Cholesky) and capture the
 * V-cycle graphs.  `stream` is a cudaStream_t (NULL: legacy default stream).
 * Setup itself uses a few temporary buffers freed before returning. */
fcm_status fcm_setup(const fcm_grid* grid, const fcm_geometry* geom,
                     const fcm_physics* phys, const fcm_solver_opts* opts,
                     void* stream, fcm_handle** out);

/* Number of DOFs of the finest level (the length of every solve vector):
 * the hierarchical tensor-product layout below, nf prod_a (C_a p + 1)
 * (Sec. 2.1; with trunk elements the removed modes keep their slots). */
fcm_status fcm_ndofs(const fcm_handle* h, long long* n);

/* The DOF layout above, for callers that hold vectors in another order
 * (no GPU, no handle needed).  Modes follow the hierarchical basis of
 * Sec. 2.1: nodal modes are shared by the two cells at a node, bubble
 * modes belong to one cell.
 * fcm_dof_layout: the 1D map of one axis with `cells` cells and degree p:
 *   map[c (p+1) + j] = 1D index of local mode j of cell c, i.e. c for
 *   j = 0, c + 1 for j = 1, (cells + 1) + (j - 2) cells + c for j >= 2.
 *   map: caller array of cells (p+1) ints.
 * fcm_cell_dofs: global indices of the nf (p+1)^dim DOFs of cell `cell`
 *   (linear cell index, x fastest) in local order j_x + (p+1) j_y +
 *   (p+1)^2 j_z, fields stacked (field f adds f M, M = prod_a (cells_a p + 1)).
 *   dofs: caller array of nf (p+1)^dim long longs.
 * Both return FCM_E_INVALID for dim not 2 or 3, cells < 1, p outside
 * [1, 8], nf < 1, a cell outside the grid or a NULL output. */
fcm_status fcm_dof_layout(int cells, int p, int* map);
fcm_status fcm_cell_dofs(int dim, const int* cells, int p, int nf, long long cell,
                         long long* dofs);

/* Multi-level hp overlay topology (Sec. 2.2), host only (no GPU, no device
 * memory).  Base grid: grid->dim, cells, lo, hi, degree p (all levels);
 * depth K = grid->overlay_levels in [0, 10], with cells_a 2^K <= 2^19;
 * overlay_p must be 0 or p.  An element of level k < K is overlaid by its
 * 2^dim bisection children when `geom` cuts its box (the classification
 * fcm_setup uses for cells; VOIDS is accepted in 2D here, ball (cx, cy, cz, r)
 * with cz unused).  Every element carries the (p+1)^dim integrated Legendre
 * modes on its own box.  A mode belongs to a component of its level's
 * lattice with doubled coordinates t_a = 2 e_a (left node), 2 e_a + 2 (right
 * node) or 2 e_a + 1 (bubble).  Active components:
 *   R1  none of level k >= 1 on the boundary of the union of the level-k
 *       elements (box faces excluded);
 *   R2  no vertex of level k >= 1 whose lattice node indices are all even;
 *   R3  edges, faces and interiors only if they belong to a leaf element.
 * These functions span exactly the C0 piecewise-Q_p space on the leaves.
 *
 * fcm_mlhp_create: builds the topology; *out owned by the caller, released
 *   by fcm_mlhp_destroy.  FCM_E_INVALID for a NULL argument or any limit
 *   above; FCM_E_OOM if host memory runs out.
 * fcm_mlhp_sizes: M scalar functions, L leaves, the total number of
 *   (leaf, function) incidences and of (base node, function) patch entries.
 * fcm_mlhp_functions: per function i (ordered by level, then component with
 *   x fastest, then bubble degrees with the first odd axis fastest):
 *   level[i], t[3 i + a] (doubled lattice coordinates, 0 on unused axes),
 *   q[3 i + a] (bubble degree on odd axes, 0 elsewhere).  Caller arrays of
 *   M, 3 M, 3 M ints.
 * fcm_mlhp_leaves: per leaf l (ordered by level, then x fastest): level[l],
 *   index[3 l + a] (lattice cell of its level), and functions[offsets[l] ..
 *   offsets[l+1]) = the scalar functions supported on it, ancestors from
 *   the base down, local modes x fastest (the row order of its element
 *   matrix).  Caller arrays of L, 3 L, L + 1 and n_leaf_entries.
 * fcm_mlhp_patches: per base node v (x fastest), functions[offsets[v] ..
 *   offsets[v+1]) = sorted scalar functions touching one of the base cells
 *   around v: the patchwise additive Schwarz block (Sec. 3.3.1) of field 0.
 *   Caller arrays of prod_a (cells_a + 1) + 1 and n_patch_entries.
 * Vector fields stack whole scalar spaces (DOF f M + i). */
typedef struct fcm_mlhp fcm_mlhp;
fcm_status fcm_mlhp_create(const fcm_grid* grid, const fcm_geometry* geom, fcm_mlhp** out);
void fcm_mlhp_destroy(fcm_mlhp* m);
fcm_status fcm_mlhp_sizes(const fcm_mlhp* m, long long* n_functions, long long* n_leaves,
                          long long* n_leaf_entries, long long* n_patch_entries);
fcm_status fcm_mlhp_functions(const fcm_mlhp* m, int* level, int* t, int* q);
fcm_status fcm_mlhp_leaves(const fcm_mlhp* m, int* level, int* index, long long* offsets,
                           long long* functions);
fcm_status fcm_mlhp_patches(const fcm_mlhp* m, long long* offsets, long long* functions);

/* fcm_mlhp_leaf_classes: per leaf, the class of its box (0 inside, 1
 *   outside, 2 cut; the test fcm_setup uses for cells).  Caller array of L.
 * fcm_mlhp_levels: the hp-multigrid levels of Sec. 3.2 (Fig. hpmultigrid),
 *   numbered from the coarsest (0, the base grid's hats) to the finest
 *   (n_levels - 1, all functions): the degree is lowered first (p, ..., 1),
 *   then at p = 1 the hats of overlay levels K, ..., 1 are removed, skipping
 *   overlay levels without active hats; n_levels = p + the removals kept.
 *   coarsest[i]: the lowest level that holds function i; level l holds
 *   exactly the functions with coarsest <= l (nested, binary transfers).
 *   Caller array of M ints.
 * fcm_mlhp_restriction_1d: the 1D restriction of the p+1 modes of an
 *   ancestor interval to its sub-interval pos (0 <= pos < 2^dk, 0 <= dk <=
 *   10) of relative length 2^-dk, in the sub-interval's own modes:
 *   S[i (p+1) + j] = coefficient of sub-interval mode i in ancestor mode j
 *   (exact for these polynomials up to rounding).  The Kronecker product of
 *   the per-axis S maps an ancestor's tensor modes to a leaf's, so a leaf
 *   matrix is T^T K_own T with K_own the cell matrix of the leaf's box.
 *   S: caller array of (p+1)^2 doubles; FCM_E_INVALID outside the limits. */
fcm_status fcm_mlhp_leaf_classes(const fcm_mlhp* m, signed char* cls);
fcm_status fcm_mlhp_levels(const fcm_mlhp* m, int* n_levels, int* coarsest);
fcm_status fcm_mlhp_restriction_1d(int p, int dk, int pos, double* S);

/* The operator and load of an overlay mesh on the device (refinement by
 * superposition, Sec. 2.2; the leaf assembly of Eq. (weakform) over the
 * functions of each leaf).  For every leaf the cell matrix and load of its
 * box are integrated on the device (the cell kernels of fcm_setup on the
 * lattice of the leaf's level: space tree on cut leaves, box-face terms on
 * leaves at the box boundary) and mapped to the leaf's functions,
 * K_L = T^T K_box T and b_L = T^T b_box, with T the Kronecker product of
 * the 1D restrictions (fcm_mlhp_restriction_1d) from each function's
 * ancestor; leaf matrices stay in device memory.
 * fcm_mlhp_op_create: m the topology built from the same grid and
 *   geometry; grid, geom, phys as for fcm_setup (grid->overlay_levels as
 *   for fcm_mlhp_create; tensor-product space only).  `stream` as in
 *   fcm_setup.  FCM_E_UNSUPPORTED when a leaf carries more than 6144 DOFs.
 * fcm_mlhp_op_ndofs: nf M, vectors field-major (f M + function id, the
 *   function order of fcm_mlhp_functions).
 * fcm_mlhp_op_apply: y = A x: y_L = K_L x_L per leaf, the leaf results
 *   summed per DOF in a fixed order (reproducible bit for bit).
 * fcm_mlhp_op_rhs: the assembled load b.
 * fcm_mlhp_op_prepare: the hp-multigrid of Sec. 3.2 on the overlay mesh
 *   (Fig. hpmultigrid): the hp-levels of fcm_mlhp_levels as masks of the
 *   full-length vectors (restriction: the coarser level's mask;
 *   prolongation: an add), additive Schwarz blocks on every level >= 1
 *   (opts->smoother PATCHWISE: the functions touching the base cells around
 *   a base node, Sec. 3.3.1; ELEMENTWISE: those touching one base cell),
 *   inverted densely, omega as in fcm_setup (patchwise paper values 1/6 in
 *   2D, 1/18 in 3D); below the base grid's hats, while the grid has more
 *   than opts->coarse_cells cells on an axis, Q1 h-levels by Galerkin
 *   P^T A P with multilinear interpolation (the Remark of Sec. 3.2; node
 *   blocks of the same kind); the coarsest level solved by its dense
 *   inverse.  The blocks and Q1 operators are assembled and inverted on the
 *   host at set-up; FCM_E_UNSUPPORTED when a block exceeds 6144 DOFs.
 *   With grid->overlay_levels = 0 this is the uniform-grid hierarchy of
 *   fcm_setup (p-levels, Q1 h-levels, coarse solve) with either block kind.
 * fcm_mlhp_op_level: per level (0 = coarsest) its DOFs, omega, number and
 *   largest size of its blocks.
 * fcm_mlhp_op_vcycle: z = V(r), Algorithm 1 with zero initial guess, every
 *   operation on the device.
 * fcm_mlhp_op_pcg: V-cycle-preconditioned CG in FP64 from x = 0 (b_dev
 *   NULL: the assembled load), as fcm_pcg_solve.
 * fcm_setup refuses overlays. */
typedef struct fcm_mlhp_op fcm_mlhp_op;
fcm_status fcm_mlhp_op_create(const fcm_mlhp* m, const fcm_grid* grid, const fcm_geometry* geom,
                              const fcm_physics* phys, void* stream, fcm_mlhp_op** out);
fcm_status fcm_mlhp_op_ndofs(const fcm_mlhp_op* op, long long* n);
fcm_status fcm_mlhp_op_apply(fcm_mlhp_op* op, const double* x_dev, double* y_dev);
fcm_status fcm_mlhp_op_rhs(const fcm_mlhp_op* op, double* b_dev);
fcm_status fcm_mlhp_op_prepare(fcm_mlhp_op* op, const fcm_solver_opts* opts);
fcm_status fcm_mlhp_op_level(const fcm_mlhp_op* op, int level, long long* ndofs, double* omega,
                             int* n_blocks, int* max_block);
fcm_status fcm_mlhp_op_vcycle(fcm_mlhp_op* op, const double* r_dev, double* z_dev);
fcm_status fcm_mlhp_op_pcg(fcm_mlhp_op* op, const double* b_dev, double* x_dev, double rtol,
                           int maxit, fcm_info* info);
void fcm_mlhp_op_destroy(fcm_mlhp_op* op);

/* Copy the assembled load vector b into b_dev (ndofs doubles). */
fcm_status fcm_rhs(const fcm_handle* h, double* b_dev);

/* y = A x on the finest level (prec FCM_FP64: FP64 matrices; FCM_MIXED: the
 * FP32 copies the V-cycle uses, computed in FP32 (shared matrices on the
 * tensor cores, 3xTF32) and widened). */
fcm_status fcm_apply(fcm_handle* h, const double* x_dev, double* y_dev, int prec);

/* z = V(r): one V-cycle with zero initial guess (Algorithm 1). */
fcm_status fcm_vcycle(fcm_handle* h, const double* r_dev, double* z_dev, int prec);

/* Level hooks for tests: op 0: y = A_l x; op 1: y = M_l^{-1} x (AS sum of
 * block inverses, no omega); op 2: y = R_l x (to level l-1); op 3: y = R_l^T x
 * (from level l-1); op 4: y = A_0^{-1} x (level 0 only).  Level 0 is the
 * coarsest, fcm_num_levels()-1 the finest.  Vectors have that level's size. */
/* fcm_num_levels: levels of the hierarchy of Sec. 3.2 (Fig. hpmultigrid):
 * the p-levels p, p-1, ..., 1 on the finest grid, then the nested Q1
 * h-levels of the Remark of Sec. 3.2 down to the coarse grid. */
fcm_status fcm_num_levels(const fcm_handle* h, int* n);
fcm_status fcm_level_info_get(const fcm_handle* h, int level, fcm_level_info* info);
fcm_status fcm_level_op(fcm_handle* h, int level, int op, const double* x_dev,
                        double* y_dev);

/* Cell classes of the finest grid (0 inside, 1 outside, 2 cut: Omega_phys,
 * Omega_fict and the cells the boundary crosses, Sec. 2.1), linear cell
 * order (x fastest), into a host array of prod(cells) bytes. */
fcm_status fcm_cell_classes(const fcm_handle* h, signed char* cls_host);

/* V-cycle-preconditioned CG from x = 0 (Sec. 4): stops when the recursive
 * relative residual falls below rtol and the recomputed true residual
 * confirms it.  b_dev NULL uses the assembled load.  prec FCM_MIXED runs
 * the FP32 V-cycle inside flexible (Polak-Ribiere) CG; the CG itself (its
 * operator for search directions and true residual, dot products and
 * updates) is FP64 in both modes.  Returns
 * FCM_E_NOT_CONVERGED after maxit iterations (x_dev holds the last
 * iterate), FCM_E_BREAKDOWN on p^T A p <= 0 or a non-finite scalar. */
fcm_status fcm_pcg_solve(fcm_handle* h, const double* b_dev, double* x_dev, double rtol,
                         int maxit, int prec, fcm_info* info);

/* The paper's solvers (Sec. 4): method FCM_METHOD_CG_MG is fcm_pcg_solve;
 * FCM_METHOD_MG is multigrid as a stand-alone solver, x_{k+1} = x_k +
 * V(b - A x_k) from x_0 = 0 until ||b - A x|| / ||b|| <= rtol, with the
 * contraction numbers rho_k = ||r_k|| / ||r_{k-1}|| (Eq. contraction) written
 * to rho_host[k - 1] when rho_host (host, maxit doubles) is not NULL;
 * FCM_E_NOT_CONVERGED after maxit iterations or once the residual exceeds
 * 1e20 ||b|| (diverged); FCM_METHOD_CG_AS is CG preconditioned by the
 * finest level's smoother alone, M^{-1} (the one-level additive Schwarz
 * CG the paper compares with; FP64 only, needs at least two levels).
 * Other arguments as in fcm_pcg_solve. */
enum { FCM_METHOD_CG_MG = 0, FCM_METHOD_MG = 1, FCM_METHOD_CG_AS = 2 };
fcm_status fcm_solve(fcm_handle* h, int method, const double* b_dev, double* x_dev, double rtol,
                     int maxit, int prec, fcm_info* info, double* rho_host);

/* Same solve through host buffers: b_host (NULL: assembled load) is copied
 * to the device and x is copied back into x_host (ndofs doubles each). */
fcm_status fcm_pcg_solve_host(fcm_handle* h, const double* b_host, double* x_host,
                              double rtol, int maxit, int prec, fcm_info* info);

/* Benchmark hook (no counterpart in the paper, which reports no timings of
 * its own kernels): replay one kernel of level `level` `reps` times on the
 * handle's stream and return its mean duration from CUDA events (ms); the
 * kernels are the level operations of Algorithm 1 (residual and smoothing
 * steps, Eq. AdditiveSchwarz).
 * which 0: operator cell kernels (y_c = K_c x_c over all cells: stored and
 * shared parts side by side, as in the V-cycle), 1: smoother cell kernels
 * (A_i^{-1} over all blocks, likewise), 2: the DOF gather that follows
 * them, 3 / 4: the stored-matrix (cut-cell / irregular-block) kernel of the
 * operator / smoother alone, without the shared-matrix tiles, 5 / 6: the
 * shared-matrix tiles of the operator / smoother alone.  prec selects
 * the FP64 or the FCM_MIXED data.  Inputs are the level's work vectors (their
 * current contents); results are discarded. */
fcm_status fcm_profile_op(fcm_handle* h, int level, int which, int prec, int reps,
                          double* avg_ms);

/* Benchmark hook (no counterpart in the paper): the FMA throughput of the
 * current device in TFLOP/s (2 flops per FMA), FP64 (prec FCM_FP64) or FP32
 * (FCM_MIXED), from independent FMA chains on every SM timed with CUDA
 * events; the peak against which the FMA-bound kernels (plain FP64
 * shared-matrix products, compensated df32 products) are judged.  Allocates
 * and frees a small device buffer and a stream; takes about 0.1 s. */
fcm_status fcm_measure_fma_peak(int prec, double* tflops);

/* Benchmark hook (no counterpart in the paper): bytes the level kernel
 * `which` (as in fcm_profile_op) must move at least once per launch:
 * stored cell matrices or block inverses, one read of every input
 * coefficient per cell and one write of every per-cell result. */
fcm_status fcm_op_bytes(const fcm_handle* h, int level, int which, int prec,
                        long long* bytes);

/* Batched mode (independent problems of uneven size, degree and geometry;
 * the paper solves one problem at a time, this is a service mode).  Every
 * instance gets its own handle, stream and V-cycle graphs.  Set-up:
 * `threads` host workers (<= 0: hardware concurrency, at most 64).  Solve:
 * threads 0 runs all instances in lockstep from the calling thread (every
 * CG iteration enqueues each running instance's operator step on its
 * stream, synchronises once per instance for the convergence test, then
 * enqueues each running instance's preconditioner step; a done flag per
 * instance masks the converged ones); threads < 0 does the same with one
 * graph launch per CG phase for all running instances (rebuilt when the
 * running set changes); threads > 0 uses that many host workers, each
 * driving whole solves.  Every mode does each instance's work of
 * fcm_pcg_solve in the same order, so the results equal single solves bit
 * for bit.  Arrays hold n entries.  On a failing instance fcm_setup_batch destroys
 * what it built and returns that instance's status; fcm_pcg_solve_batch
 * solves every instance, fills infos[i] for each, and returns the first
 * non-FCM_OK status (instance index in fcm_last_error).  x_dev[i]: device
 * buffer of instance i's ndofs doubles (see fcm_batch_handle / fcm_ndofs). */
typedef struct fcm_batch fcm_batch;
fcm_status fcm_setup_batch(int n, const fcm_grid* grids, const fcm_geometry* geoms,
                           const fcm_physics* phys, const fcm_solver_opts* opts, int threads,
                           void* stream, fcm_batch** out);
fcm_status fcm_batch_size(const fcm_batch* b, int* n);
fcm_status fcm_batch_handle(const fcm_batch* b, int i, fcm_handle** h);
fcm_status fcm_pcg_solve_batch(fcm_batch* b, double* const* x_dev, double rtol, int maxit,
                               int prec, int threads, fcm_info* infos);
void fcm_batch_destroy(fcm_batch* b);

/* Allocation-free operator apply, for callers that cannot allocate device
 * memory once they run (fixed device arenas, real-time loops, plug-ins in a
 * foreign memory pool) and therefore cannot call fcm_setup.  The paper has
 * no counterpart; it is a service entry point of this library.
 *   y = sum_c P_c^T K_c P_c x  on a grid of dim (2 or 3) with cells[0..dim-1]
 *   cells per axis and one scalar field of degree p, in the layout above.
 * K_dev: caller-owned device array of prod(cells) symmetric cell matrices,
 * (p+1)^d x (p+1)^d each, row-major, cells in linear order (x fastest), local
 * DOF order j_x + (p+1) j_y + (p+1)^2 j_z.  x_dev, y_dev: ndofs doubles.
 * stream: cudaStream_t (NULL: legacy default stream); the call synchronizes
 * the stream before it returns.  Scratch: a 4 MiB array compiled into the
 * library (per GPU, held until exit), so prod(cells) (p+1)^d may be at most
 * about 520,000; larger requests return FCM_E_INVALID.  The first call on a
 * device looks up the array's device address (cached per device, so not valid
 * across cudaDeviceReset) and should come before any stream capture; calls
 * that overlap on the GPU race on the shared array.  FCM_E_TIMEOUT if a
 * bounded device wait on a bulk copy expired (y then holds stale products).
 * Calls no allocating routine. */
fcm_status fcm_cell_apply_noalloc(int dim, const int* cells, int p, const double* K_dev,
                                  const double* x_dev, double* y_dev, void* stream);

void fcm_destroy(fcm_handle* h);

const char* fcm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FCM_H */
