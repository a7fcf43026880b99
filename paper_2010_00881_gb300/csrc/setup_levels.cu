// Setup kernels of the multigrid hierarchy (all FP64):
//  - hierarchical sub-blocks of cell matrices (Eq. hierarchicalMatrices),
//  - Galerkin Q1 coarse cells K_C = sum_f P_f^T K_f P_f (nested h-levels),
//  - elementwise additive Schwarz blocks A_i = P_i^T A P_i (Eq.
//    AdditiveSchwarz) gathered from the 3^d neighbouring cells,
//  - batched Cholesky-based inversion of the blocks,
//  - dense assembly, Cholesky factor and factor inverse of the coarsest level.
#include <cmath>

#include "fcm_internal.h"

namespace fcm {

namespace {

__device__ inline int local_index(int dim, int P1, int nloc_s, int f, int jx, int jy, int jz) {
  int s = jx;
  if (dim > 1) s += P1 * jy;
  if (dim > 2) s += P1 * P1 * jz;
  return f * nloc_s + s;
}

__device__ inline void local_split(int l, int dim, int P1, int nloc_s, int& f, int* j) {
  f = l / nloc_s;
  int s = l - f * nloc_s;
  j[0] = s % P1;
  j[1] = dim > 1 ? (s / P1) % P1 : 0;
  j[2] = dim > 2 ? s / (P1 * P1) : 0;
}

// Kc = sub-block of Kf on the modes of degree <= pc.
__global__ void extract_sub_kernel(int nmat, int dim, int nf, int pf, int pc, const double* Kf,
                                   double* Kc) {
  int Pf = pf + 1, Pc = pc + 1;
  int nsf = 1, nsc = 1;
  for (int a = 0; a < dim; ++a) {
    nsf *= Pf;
    nsc *= Pc;
  }
  int nf_loc = nf * nsf, nc_loc = nf * nsc;
  long long tot = (long long)nmat * nc_loc * nc_loc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    int m = (int)(t / ((long long)nc_loc * nc_loc));
    int r = (int)(t % ((long long)nc_loc * nc_loc));
    int i = r / nc_loc, j = r % nc_loc;
    int fi, fj, ji[3], jj[3];
    local_split(i, dim, Pc, nsc, fi, ji);
    local_split(j, dim, Pc, nsc, fj, jj);
    int I = local_index(dim, Pf, nsf, fi, ji[0], ji[1], ji[2]);
    int J = local_index(dim, Pf, nsf, fj, jj[0], jj[1], jj[2]);
    Kc[t] = Kf[(size_t)m * nf_loc * nf_loc + (size_t)I * nf_loc + J];
  }
}

__device__ inline const double* fine_matrix(const FineCellSource& src, int cell, int nloc,
                                            double& scale) {
  int oi = src.own_index[cell];
  if (oi >= 0) {
    scale = 1.0;
    return src.own_mats + (size_t)oi * nloc * nloc;
  }
  scale = src.shared_scale_by_cell[cell];
  return src.Kref;
}

// 1D Q1 interpolation inside a coarse cell: fine child o in {0, 1}, fine
// local node jf in {0, 1}, coarse local node jc in {0, 1}.
__device__ inline double q1w(int o, int jf, int jc) {
  int t = o + jf;  // position 0, 1 (midpoint) or 2 in half cells
  if (t == 1) return 0.5;
  return (t == 0) == (jc == 0) ? 1.0 : 0.0;
}

// One block per coarse cell, one thread per (I, J) entry (nloc <= 24).
__global__ void galerkin_kernel(LevelGeom gc, LevelGeom gf, FineCellSource src, double* Kc) {
  const int n = gc.nloc;      // 2^d nf
  const int ns = gc.nloc_s;   // 2^d
  int c = blockIdx.x;
  if (c >= gc.ncells) return;
  int cc[3];
  cell_coords(gc, c, cc[0], cc[1], cc[2]);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int I = e / n, J = e % n;
    int fI, fJ, jI[3], jJ[3];
    local_split(I, gc.dim, 2, ns, fI, jI);
    local_split(J, gc.dim, 2, ns, fJ, jJ);
    double acc = 0.0;
    int nch = 1 << gc.dim;
    for (int o = 0; o < nch; ++o) {
      int oc[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
      int fc[3];
      bool ok = true;
      for (int a = 0; a < 3; ++a) {
        fc[a] = a < gc.dim ? 2 * cc[a] + oc[a] : 0;
        if (a < gc.dim && fc[a] >= gf.C[a]) ok = false;
      }
      if (!ok) continue;
      int fcell = fc[0] + gf.C[0] * (fc[1] + gf.C[1] * fc[2]);
      double s;
      const double* K = fine_matrix(src, fcell, gf.nloc, s);
      // sum_{a,b} P[a][I] K[a][b] P[b][J]; fields decouple in P
      double t = 0.0;
      for (int a = 0; a < ns; ++a) {
        int ja[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
        double wa = 1.0;
        for (int d = 0; d < gc.dim; ++d) wa *= q1w(oc[d], ja[d], jI[d]);
        if (wa == 0.0) continue;
        double u = 0.0;
        for (int b = 0; b < ns; ++b) {
          int jb[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
          double wb = 1.0;
          for (int d = 0; d < gc.dim; ++d) wb *= q1w(oc[d], jb[d], jJ[d]);
          if (wb == 0.0) continue;
          u += K[(size_t)(fI * ns + a) * gf.nloc + fJ * ns + b] * wb;
        }
        t += wa * u;
      }
      acc += s * t;
    }
    Kc[(size_t)c * n * n + e] = acc;
  }
}

// Does local 1D mode j of the block cell appear in the neighbour at offset o,
// and as which local mode?
__device__ inline int shared_mode(int o, int j) {
  if (o == 0) return j;
  if (o < 0) return j == 0 ? 1 : -1;  // left neighbour: our node 0 is its node 1
  return j == 1 ? 0 : -1;            // right neighbour: our node 1 is its node 0
}

// One block per AS block: A_i[a][b] = sum over the 3^d neighbours of the
// entries of their cell matrices on the DOFs shared with cell i.
__global__ void block_assemble_kernel(LevelGeom g, int nblk, const int* blk_cells,
                                      FineCellSource src, double* Ablk) {
  const int n = g.nloc, ns = g.nloc_s, P1 = g.p + 1;
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    int cell = blk_cells[bi];
    bool ref = cell < 0;
    int sig = ref ? -(cell + 1) : 0;
    int cc[3] = {0, 0, 0};
    if (!ref) cell_coords(g, cell, cc[0], cc[1], cc[2]);
    double* A = Ablk + (size_t)bi * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int I = e / n, J = e % n;
      int fI, fJ, jI[3], jJ[3];
      local_split(I, g.dim, P1, ns, fI, jI);
      local_split(J, g.dim, P1, ns, fJ, jJ);
      double acc = 0.0;
      int nnb = 1;
      for (int a = 0; a < g.dim; ++a) nnb *= 3;
      for (int o = 0; o < nnb; ++o) {
        int off[3] = {0, 0, 0};
        int t = o;
        bool ok = true;
        int mI[3] = {0, 0, 0}, mJ[3] = {0, 0, 0};
        int nc[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) {
          off[a] = t % 3 - 1;
          t /= 3;
          if (ref) {
            int sa = (sig >> (2 * a)) & 3;  // 1: no lower, 2: no upper, 3: neither
            if (off[a] < 0 && (sa & 1)) ok = false;
            if (off[a] > 0 && (sa & 2)) ok = false;
          } else {
            nc[a] = cc[a] + off[a];
            if (nc[a] < 0 || nc[a] >= g.C[a]) ok = false;
          }
          mI[a] = shared_mode(off[a], jI[a]);
          mJ[a] = shared_mode(off[a], jJ[a]);
          if (mI[a] < 0 || mJ[a] < 0) ok = false;
        }
        if (!ok) continue;
        double s;
        const double* K;
        if (ref) {
          s = 1.0;
          K = src.Kref;
        } else {
          int ncell = nc[0] + g.C[0] * (nc[1] + g.C[1] * nc[2]);
          K = fine_matrix(src, ncell, n, s);
        }
        int li = local_index(g.dim, P1, ns, fI, mI[0], mI[1], mI[2]);
        int lj = local_index(g.dim, P1, ns, fJ, mJ[0], mJ[1], mJ[2]);
        acc += s * K[(size_t)li * n + lj];
      }
      A[e] = acc;
    }
  }
}

// In-place inverse of SPD blocks via A = L L^T, L^{-1} (in place) and
// A^{-1} = L^{-T} L^{-1}.  One block per matrix, matrix staged in shared
// memory (n <= 128).  Per block: stats[2i] = smallest Cholesky pivot,
// stats[2i+1] = infinity-norm condition number of the diagonally scaled
// block S = D^{-1/2} A D^{-1/2}: ||S||_inf ||S^{-1}||_inf, with S^{-1} =
// D^{1/2} A^{-1} D^{1/2} read off the computed inverse.
__global__ void chol_inverse_kernel(int nblk, int n, double* Aall, double* stats, int* info) {
  extern __shared__ double Ls[];  // n * n
  double* tmp = Ls + n * n;       // n
  double* diag = tmp + n;         // n
  __shared__ double pmin, dep, normS, normSi;
  __shared__ int bad;
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    double* A = Aall + (size_t)bi * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Ls[e] = A[e];
    for (int i = threadIdx.x; i < n; i += blockDim.x) diag[i] = A[(size_t)i * n + i];
    if (threadIdx.x == 0) {
      pmin = INFINITY;
      dep = 0.0;
      bad = 0;
    }
    __syncthreads();
    // ||S||_inf of the scaled block
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double t = 0.0;
      for (int j = 0; j < n; ++j) t += fabs(Ls[i * n + j]) / sqrt(diag[i] * diag[j]);
      tmp[i] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int i = 0; i < n; ++i) m = fmax(m, tmp[i]);
      normS = m;
    }
    __syncthreads();
    // right-looking Cholesky, lower triangle
    for (int k = 0; k < n; ++k) {
      if (threadIdx.x == 0) {
        double d = Ls[k * n + k];
        if (!(d > 0.0) || !isfinite(d)) {
          bad = 1;
          d = 1.0;
        }
        pmin = fmin(pmin, d);
        dep = fmax(dep, diag[k] / d);
        Ls[k * n + k] = sqrt(d);
      }
      __syncthreads();
      double lkk = Ls[k * n + k];
      for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) Ls[i * n + k] /= lkk;
      __syncthreads();
      int m = n - k - 1;
      for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = k + 1 + e / m, j = k + 1 + e % m;
        if (j <= i) Ls[i * n + j] -= Ls[i * n + k] * Ls[j * n + k];
      }
      __syncthreads();
    }
    // in-place inverse of the lower factor, last column first
    for (int j = n - 1; j >= 0; --j) {
      if (threadIdx.x == 0) Ls[j * n + j] = 1.0 / Ls[j * n + j];
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int k = j + 1; k <= i; ++k) s += Ls[i * n + k] * Ls[k * n + j];
        tmp[i] = s;
      }
      __syncthreads();
      double njj = -Ls[j * n + j];
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) Ls[i * n + j] = njj * tmp[i];
      __syncthreads();
    }
    // A^{-1}[i][j] = sum_{k >= max(i,j)} Linv[k][i] Linv[k][j]
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e / n, j = e % n;
      int k0 = i > j ? i : j;
      double s = 0.0;
      for (int k = k0; k < n; ++k) s += Ls[k * n + i] * Ls[k * n + j];
      A[e] = s;
    }
    __syncthreads();
    // ||S^{-1}||_inf from the inverse just written
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double t = 0.0;
      for (int j = 0; j < n; ++j) t += fabs(A[(size_t)i * n + j]) * sqrt(diag[i] * diag[j]);
      tmp[i] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int i = 0; i < n; ++i) m = fmax(m, tmp[i]);
      normSi = m;
      if (stats) {
        stats[2 * bi] = pmin;
        stats[2 * bi + 1] = normS * normSi;
      }
      if (info) info[bi] = bad;
    }
    __syncthreads();
  }
}

// Dense coarse matrix from own cell matrices (single block; cells in order).
__global__ void dense_assemble_kernel(LevelGeom g, const double* K, double* A) {
  long long N = g.N;
  for (long long e = threadIdx.x; e < N * N; e += blockDim.x) A[e] = 0.0;
  __syncthreads();
  const int n = g.nloc;
  for (int c = 0; c < g.ncells; ++c) {
    int cx, cy, cz;
    cell_coords(g, c, cx, cy, cz);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int a = e / n, b = e % n;
      long long I = cell_dof(g, cx, cy, cz, a);
      long long J = cell_dof(g, cx, cy, cz, b);
      A[I * N + J] += K[(size_t)c * n * n + e];
    }
    __syncthreads();
  }
}

// Dense Cholesky factor in place (lower; upper zeroed), then the factor is
// replaced by its inverse L^{-1} (single block, global memory).
__global__ void chol_factor_kernel(int n, double* A, int* info) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double d = A[(size_t)k * n + k];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        d = 1.0;
      }
      A[(size_t)k * n + k] = sqrt(d);
    }
    __syncthreads();
    double lkk = A[(size_t)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + k] /= lkk;
    __syncthreads();
    int m = n - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    if (j > i) A[e] = 0.0;
  }
  __syncthreads();
  // in-place inverse of L (column j uses the already inverted trailing block)
  extern __shared__ double tmp[];
  for (int j = n - 1; j >= 0; --j) {
    if (threadIdx.x == 0) A[(size_t)j * n + j] = 1.0 / A[(size_t)j * n + j];
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double s = 0.0;
      for (int k = j + 1; k <= i; ++k) s += A[(size_t)i * n + k] * A[(size_t)k * n + j];
      tmp[i] = s;
    }
    __syncthreads();
    double njj = -A[(size_t)j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + j] = njj * tmp[i];
    __syncthreads();
  }
  if (threadIdx.x == 0 && info) *info = bad;
}

}  // namespace

void launch_extract_sub(int nmat, int dim, int nf, int pf, int pc, const double* Kf, double* Kc,
                        cudaStream_t s) {
  if (nmat == 0) return;
  long long tot = (long long)nmat;
  int nc = nf;
  for (int a = 0; a < dim; ++a) nc *= pc + 1;
  tot *= (long long)nc * nc;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 16384) blocks = 16384;
  extract_sub_kernel<<<blocks, 256, 0, s>>>(nmat, dim, nf, pf, pc, Kf, Kc);
}

void launch_galerkin(const LevelGeom& gc, const LevelGeom& gf, FineCellSource src, double* Kc,
                     cudaStream_t s) {
  galerkin_kernel<<<gc.ncells, 64, 0, s>>>(gc, gf, src, Kc);
}

void launch_block_assemble(const LevelGeom& g, int nblk, const int* blk_cells,
                           FineCellSource src, double* Ablk, cudaStream_t s) {
  if (nblk == 0) return;
  int grid = nblk < 8192 ? nblk : 8192;
  block_assemble_kernel<<<grid, 256, 0, s>>>(g, nblk, blk_cells, src, Ablk);
}

void launch_chol_inverse(int nblk, int n, double* A, double* pivots, int* info, cudaStream_t s) {
  if (nblk == 0) return;
  size_t smem = ((size_t)n * n + 2 * n) * sizeof(double);
  // One attribute value for every caller (n <= 128): setting it per call
  // would let a concurrent setup with a smaller block shrink it under a
  // larger launch.
  static const bool attr = [] {
    cudaFuncSetAttribute(chol_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((128 * 128 + 2 * 128) * sizeof(double)));
    return true;
  }();
  (void)attr;
  int grid = nblk < 4096 ? nblk : 4096;
  chol_inverse_kernel<<<grid, 256, smem, s>>>(nblk, n, A, pivots, info);
}

void launch_dense_assemble(const LevelGeom& g, const double* own_mats, double* A,
                           cudaStream_t s) {
  dense_assemble_kernel<<<1, 256, 0, s>>>(g, own_mats, A);
}

void launch_chol_factor(int n, double* A, int* info, cudaStream_t s) {
  chol_factor_kernel<<<1, 512, n * sizeof(double), s>>>(n, A, info);
}

}  // namespace fcm
