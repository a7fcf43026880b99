// Internal declarations of the GB300 FCM multigrid library (not part of the
// C ABI).  Layout conventions follow include/fcm.h: hierarchical per-axis 1D
// indices (nodes, then bubbles by degree), x fastest, fields stacked.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fcm.h"

namespace fcm {

constexpr int kMaxP = 8;
constexpr int kMaxDepth = 4;

// Geometry of one multigrid level as seen by the kernels.
// n / d for 0 <= n < 2^31 and 1 <= d < 2^31 by a multiply-high and a shift
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): with s = ceil(log2 d) and
// mul = floor(2^32 (2^s - d) / d) + 1, n / d = (mulhi(n, mul) + n) >> s.
struct FastDiv {
  unsigned mul;
  int shift;
};
inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  int s = 0;
  while ((1LL << s) < d) ++s;
  f.shift = s;
  f.mul = (unsigned)((((1ULL << s) - (unsigned long long)d) << 32) / (unsigned long long)d + 1);
  return f;
}
__host__ __device__ inline int fdiv(const FastDiv& f, int n) {
#ifdef __CUDA_ARCH__
  const unsigned hi = __umulhi((unsigned)n, f.mul);
#else
  const unsigned hi = (unsigned)(((unsigned long long)(unsigned)n * f.mul) >> 32);
#endif
  return (int)((hi + (unsigned)n) >> f.shift);
}

struct LevelGeom {
  int dim, nf, p;
  int C[3];        // cells per axis (1 for unused axes)
  int m[3];        // 1D indices per axis, C p + 1 (1 for unused axes)
  long long M;     // scalar DOFs
  long long N;     // nf * M
  int nloc_s;      // (p+1)^dim
  int nloc;        // nf * nloc_s
  int ncells;
  FastDiv dC[3];   // division by C[a]
  FastDiv dm[2];   // division by m[0], m[1]
  FastDiv dM;      // division by M
};

LevelGeom make_geom(int dim, int nf, int p, const int* C);

__host__ __device__ inline int dof1(int C, int c, int j) {
  return j == 0 ? c : (j == 1 ? c + 1 : (C + 1) + (j - 2) * C + c);
}

// Global index of local DOF l of cell (cx, cy, cz).
__host__ __device__ inline long long cell_dof(const LevelGeom& g, int cx, int cy, int cz, int l) {
  int f = l / g.nloc_s;
  int s = l - f * g.nloc_s;
  int P1 = g.p + 1;
  int jx = s % P1;
  int jy = g.dim > 1 ? (s / P1) % P1 : 0;
  int jz = g.dim > 2 ? s / (P1 * P1) : 0;
  long long ix = dof1(g.C[0], cx, jx);
  long long iy = g.dim > 1 ? dof1(g.C[1], cy, jy) : 0;
  long long iz = g.dim > 2 ? dof1(g.C[2], cz, jz) : 0;
  return (long long)f * g.M + ix + (long long)g.m[0] * (iy + (long long)g.m[1] * iz);
}

__host__ __device__ inline void cell_coords(const LevelGeom& g, int c, int& cx, int& cy, int& cz) {
  cx = c % g.C[0];
  int t = c / g.C[0];
  cy = t % g.C[1];
  cz = t / g.C[1];
}

// ----------------------------------------------------------------------------
// Problem description copied from the C ABI descriptors (device-friendly).
struct Problem {
  int dim, nf, p, pde;
  int C[3];
  double lo[3], hi[3], h[3];
  int geom_kind;
  int geom_complement;          // 1: Omega_phys = {psi >= 0}
  int n_gparams;
  double* d_gparams;            // device copy of geometry parameters
  double kappa, E, nu, alpha, beta;
  int source;
  double f0, src_a;
  int dirichlet, g;
  unsigned dir_faces;
  int traction_face;
  double traction[3];
  int quad_depth;
  int sumfact;                  // 1: leaf sums by sum factorisation (FCM_QUAD_SUMFACT)
  int trunk;                    // 1: trunk-space elements (non-trunk modes removed)
  int drop;                     // 1: fully fictitious cells removed
};

// Cell classes.
enum { CLS_INSIDE = 0, CLS_OUTSIDE = 1, CLS_CUT = 2 };

// ----------------------------------------------------------------------------
// Per-level operator and smoother data (solve layout).
//
// Stored cell matrices are symmetric and kept with rows padded to `ld`
// entries (a multiple of 4) so that every row starts on a 16-byte boundary.
// Element types: the vector precision TV (FP64 path: double, mixed path:
// float) or, for the mixed path's extended-precision islands, pairs of
// floats (hi, lo) with hi = fl32(a), lo = fl32(a - hi) ("df32").
struct CellSet {
  int n = 0;                 // cells in the set
  int* cells = nullptr;      // linear cell ids (device)
  void* mats = nullptr;      // [n][nloc][ld] (device)
};

struct TileList {
  int ntiles = 0;
  int4* tiles = nullptr;     // {matrix id, start, count, 0} (device), <= 64 cells each
  int* cells = nullptr;      // cells grouped by matrix (device)
  int ncells = 0;
  int ntiles_mma = 0;        // the same cells in tiles of <= 128 (tensor-core kernel)
  int4* tiles_mma = nullptr;
};

template <typename T>
struct SharedSet {
  TileList tl;
  T* scale = nullptr;        // per entry of tl.cells
  T* mats = nullptr;         // [nmats][nloc][nloc] (canonical, unpadded)
  int nmats = 0;
  // FP32 only: the matrices as tensor-core operands, [nmats][hi, lo][NP x KD]
  // in the K-major core-matrix layout (see launch_mma_operands)
  float* mma_b = nullptr;
  // FP32 only: use the tensor cores only where the CUDA-core tiles cannot
  // run beside the stored-matrix streaming (set for the smoother's shared
  // inverses, whose many per-signature operands cost more than they gain
  // when both kernels fit side by side)
  bool mma_only_alone = false;
  // FP64 only, set when the one shared matrix is a Kronecker sum (the uncut
  // Poisson cell, Sec. 2.1): its 1D factors [axis][K1, M1][P][P] with
  // P = p + 1, K = sum_a (x)_b (K1 if a == b else M1)_b, axis x fastest
  const double* kron = nullptr;
};

// Whether the sum-factorised apply of a Kronecker-sum shared matrix
// (SharedSet::kron) is built for this dimension and degree.
bool kron_supported(int dim, int p);

// Tensor-core operand sizes of an n x n shared matrix: reduction length KD
// (n rounded up to a multiple of 8) and N extent NP (n rounded up to a
// multiple of 16, at least 16).
inline int mma_kd(int n) { return (n + 7) & ~7; }
inline int mma_np(int n) { return n <= 16 ? 16 : (n + 15) & ~15; }
// Split nmats FP32 n x n matrices into TF32 parts (hi = tf32(v), lo = v - hi)
// in the operand layout of the tensor-core kernel: out holds nmats x 2 x
// mma_np(n) x mma_kd(n) floats, zero-padded.
void launch_mma_operands(int n, int nmats, const float* mats, float* out, cudaStream_t s);

template <typename TV>
struct OpData {
  int ld = 0;                // padded row length of stored matrices
  CellSet own;               // stored matrices in precision TV
  CellSet own_x;             // FP32 vectors only: df32 matrices (islands of the mixed V-cycle)
  SharedSet<TV> sh;
};

// Padded row length of stored cell matrices.
inline int padded_ld(int n) { return (n + 3) & ~3; }

// Repack canonical FP64 n x n matrices (optionally selected by index) into
// the solve layout [count][n][ld]: kind 0 = double, 1 = float, 2 = df32.
void launch_repack(int count, int n, int ld, const double* src, const int* sel, int kind,
                   void* dst, cudaStream_t s);

// A second stream on which the shared-matrix tiles of a cell operation run
// beside the stored-matrix kernels (one is bound by FMA issue, the other by
// HBM bandwidth); `fork` and `join` order it against the main stream, also
// under stream capture, where they become parallel graph branches.
struct SideStream {
  cudaStream_t s2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

// Launch a cell operation Y[l][c] = (S_c x_c)[l] for every cell in `op`
// (Y is stored local-index-major: Y[l * ncells + cell]).  With `side`, the
// tiles run on side->s2 and the main stream waits for them before returning.
template <typename TV>
void launch_cell_op(const LevelGeom& g, const OpData<TV>& op, const TV* x, TV* Y,
                    cudaStream_t s, const SideStream* side = nullptr);

// Y[l][c] = diagonal entry l of cell c's matrix in `op` (FP64 data);
// sh_mat[j]: matrix id of the j-th shared cell (op.sh.tl.cells order).
void launch_cell_diag(const LevelGeom& g, const OpData<double>& op, const int* sh_mat,
                      double* Y, cudaStream_t s);
// Jacobi step: x = w dinv r (init) or x += w dinv r, N entries.
template <typename TV>
void launch_jacobi(long long N, const TV* dinv, const TV* r, TV* x, double w, bool init,
                   cudaStream_t s);

// Trunk space of degree q on a level of degree p: zero the rows and columns
// of the non-trunk local modes of `count` canonical n x n matrices (with a
// unit diagonal there if unit_diag, so that a block stays invertible), or
// zero the non-trunk entries of a level vector.
void launch_trunk_mask_mats(long long count, int dim, int nf, int p, int q, bool unit_diag,
                            double* mats, cudaStream_t s);
void launch_trunk_mask_vec(const LevelGeom& g, int q, double* v, cudaStream_t s);

// Node-centric operations of the levels with one mode per node and field
// (p = 1 and the Q1 h-levels: n = nf 2^d): the cell products and the DOF
// gather in one pass, every DOF summing the rows of its cells' matrices
// against their coefficients (see node_kernel).  Per cell: code >= 0
// indexes the first stored set (m1, TV precision), code <= -2 the second
// (m2: df32 pairs in the mixed path), code -1 a shared matrix mat[c]
// (canonical n x n in sh) scaled by scale[c].
template <typename TV>
struct NodeSet {
  bool ok = false;
  int ld = 0;
  const int* code = nullptr;
  const int* mat = nullptr;
  const TV* scale = nullptr;
  const void* m1 = nullptr;
  const void* m2 = nullptr;
  const TV* sh = nullptr;
};
// out = mode(sum), the gather modes below; x the cell products' input.
template <typename TV>
void launch_node(const LevelGeom& g, const NodeSet<TV>& op, const TV* x, const TV* b, TV* out,
                 double w, int mode, cudaStream_t s);

// Multi-level hp operator (mlhp_ops.cu): per-incidence restriction data
// (mlhp_inc_bytes() bytes each: table offsets and local modes, 3 + 3 ints),
// leaf matrices K_L = T^T K_box T and loads b_L = T^T b_box, the leaf-wise
// apply and the fixed-order DOF gather.
size_t mlhp_inc_bytes();
void launch_leaf_transform(int nleaf, int dim, int P1, int nf, const long long* off,
                           const void* inc, const double* S, const double* Kbox,
                           const double* bbox, const long long* koff, const long long* woff,
                           double* W, double* KL, double* bL, cudaStream_t s);
// Rows per work item of launch_leaf_apply (its block size): items are
// (leaf or block, first row), one per kLeafRows rows of each leaf.
constexpr int kLeafRows = 128;
void launch_leaf_apply(int nitem, const int2* items, int nf, long long M, int max_nl,
                       const long long* off, const long long* fn, const long long* koff,
                       const double* KL, const double* x, double* Yl, cudaStream_t s);
void launch_leaf_gather(long long M, int nf, const long long* ioff, const long long* ibase,
                        const int* istride, const double* Yl, double* out, cudaStream_t s);

// Removed DOFs (fully fictitious cells dropped): empty rows of `count`
// assembled n x n blocks get a unit diagonal (phase 0, flags written) and
// are zeroed in the inverse (phase 1); a vector's entries of removed scalar
// DOFs (keep[i % M] == 0) are zeroed.
void launch_mask_empty_rows(long long count, int n, int phase, double* mats,
                            unsigned char* flags, cudaStream_t s);
template <typename T>
void launch_mask_vec(long long N, long long M, const unsigned char* keep, T* v, cudaStream_t s);

// Level vector operations of the overlay hp-multigrid (mode 0: out = mask
// (a - b), 1: out += w a, 2: out = w a, 3: out = mask a, 4: out += a,
// 5: out = a + w out).
void launch_mlhp_vec(long long N, int mode, const unsigned char* mask, const double* a,
                     const double* b, double* out, double w, cudaStream_t s);

// Independent CG solves of several handles in lockstep from the calling
// thread (batched mode; graph: one graph launch per CG phase for all
// running instances); the first failing status in instance order.
fcm_status pcg_solve_lockstep(fcm_handle* const* hs, int n, double* const* x, double rtol,
                              int maxit, int prec, fcm_info* infos, bool graph);

// y = A x for a CSR matrix (rows x any), one thread per row.
void launch_csr_spmv(long long rows, const long long* ptr, const long long* col,
                     const double* val, const double* x, double* y, cudaStream_t s);

// DOF gather modes: out = sum | out = b - sum | out += w sum | out = w sum
enum { GATHER_SET = 0, GATHER_RESID = 1, GATHER_ADD = 2, GATHER_SCALE = 3 };
template <typename TV>
void launch_gather(const LevelGeom& g, int mode, const TV* Y, const TV* b, TV* out, double w,
                   cudaStream_t s);

template <typename TV>
void launch_p_restrict(const LevelGeom& gc, const LevelGeom& gf, const TV* rf, TV* bc,
                       cudaStream_t s);
template <typename TV>
void launch_p_prolong_add(const LevelGeom& gc, const LevelGeom& gf, const TV* xc, TV* xf,
                          cudaStream_t s);
template <typename TV>
void launch_h_restrict(const LevelGeom& gc, const LevelGeom& gf, const TV* rf, TV* bc,
                       cudaStream_t s);
template <typename TV>
void launch_h_prolong_add(const LevelGeom& gc, const LevelGeom& gf, const TV* xc, TV* xf,
                          cudaStream_t s);
// x = L^{-T} L^{-1} b with the dense lower Cholesky factor L (n x n, FP64).
template <typename TV>
void launch_coarse_solve(int n, const double* L, const TV* b, TV* x, cudaStream_t s);

// CG helpers (FP64).
constexpr int kDotBlocks = 592;  // fixed: 4 x 148, keeps reductions deterministic
void launch_dot_partials(const double* a, const double* b, long long n, double* partials,
                         cudaStream_t s);
void launch_dot2_partials(const double* a, const double* b, const double* c, long long n,
                          double* partials, cudaStream_t s);
void launch_reduce(const double* partials, int count, double* out, cudaStream_t s);
struct CGScalars {
  double rz;        // r_k^T z_k
  double pq;        // p^T A p
  double alpha, beta;
  double rr;        // ||r||^2 after the update
  double rz_new, rzold_new;
  int flag;         // nonzero: breakdown detected
};
void launch_cg_update_xr(double* x, double* r, const double* p, const double* q, long long n,
                         const double* pq_partials, CGScalars* sc, double* rr_partials,
                         cudaStream_t s);
void launch_cg_update_p(double* p, const double* z, long long n, const double* rz_partials,
                        int flexible, CGScalars* sc, cudaStream_t s);
void launch_cg_init(const double* r, const double* z, long long n, const double* rz_partials,
                    double* p, CGScalars* sc, cudaStream_t s);
void launch_copy_d2f(const double* a, float* b, long long n, cudaStream_t s);
void launch_copy_f2d(const float* a, double* b, long long n, cudaStream_t s);
void launch_axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s);
void launch_scale_copy(const double* x, double* y, double a, long long n, cudaStream_t s);
void launch_fill_sin(double* v, long long n, cudaStream_t s);
void launch_d2f_mats(const double* a, float* b, long long n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Setup kernels.
void launch_gauss_table(int n, double* nodes_weights, cudaStream_t s);
void launch_classify(const Problem& P, signed char* cls, unsigned char* faces, cudaStream_t s);
// Element matrices and loads of `ncell` own cells (cells[i] < 0: the
// reference uncut cell with alpha = 1, no surface and no faces).
void launch_element_own(const Problem& P, const double* gauss, int ncell, const int* cells,
                        double* K, double* bvec, int* leaf_scratch, int max_leaves,
                        cudaStream_t s);
// Load vectors of uncut cells: B[l][c] = alpha_c int f N_l ([local][cell]).
void launch_load_uncut(const Problem& P, const double* gauss, int ncell, const int* cells,
                       const signed char* cls, double* Bcells, cudaStream_t s);
// Scatter per-own-cell loads into the per-cell load array.
void launch_scatter_rows(int n, const int* cells, const double* src, int nloc, long long ncells,
                         double* Bcells, cudaStream_t s);
// Sub-block extraction: the level-(pc) cell matrix of a level-(pf) matrix.
void launch_extract_sub(int nmat, int dim, int nf, int pf, int pc, const double* Kf,
                        double* Kc, cudaStream_t s);
// Galerkin Q1 coarse cells.
struct FineCellSource {
  const int* own_index;      // per fine cell: index into own mats or -1
  const double* own_mats;
  const double* shared_scale_by_cell;  // per fine cell scale of K_ref when own_index < 0
  const double* Kref;
};
void launch_galerkin(const LevelGeom& gc, const LevelGeom& gf, FineCellSource src,
                     double* Kc, cudaStream_t s);
// AS block assembly for a list of blocks; cell >= 0: real cell, cell < 0:
// reference signature -(sig+1) on an all-shared grid.
void launch_block_assemble(const LevelGeom& g, int nblk, const int* blk_cells,
                           FineCellSource src, double* Ablk, cudaStream_t s);
// In-place Cholesky inverse of nblk SPD blocks; pivots[2*i] = min, [2*i+1] =
// max of diag(L)^2; info[i] != 0 on a non-positive pivot.
void launch_chol_inverse(int nblk, int n, double* A, double* pivots, int* info,
                         cudaStream_t s);
void launch_chol_factor(int n, double* A, int* info, cudaStream_t s);
void launch_dense_assemble(const LevelGeom& g, const double* own_mats, double* A,
                           cudaStream_t s);

// Kernel attributes (shared-memory limits) that must not be set while a
// stream is being captured; call before the first launch on a device.
cudaError_t prepare_kernels();

std::string cuda_msg(cudaError_t e);

// Read (and reset) the flag the streaming kernels set when a bounded wait on
// a bulk copy expired.
cudaError_t read_and_clear_timeout(int* flag, cudaStream_t s);

// Set the thread-local message returned by fcm_last_error().
void set_last_error(const char* msg);

}  // namespace fcm
