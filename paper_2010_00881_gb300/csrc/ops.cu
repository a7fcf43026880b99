// Solve-path kernels of the V-cycle and of CG.
//
// Operator apply and additive Schwarz smoothing share one pattern: for every
// cell (elementwise AS blocks are cells) gather the cell's coefficients,
// multiply by a dense cell matrix (the stiffness K_c for A, the block
// inverse A_i^{-1} for M^{-1}), and write the product into a per-cell buffer
// Y[cell][local].  A second, DOF-centric pass sums the <= 2^d contributions
// of every DOF in a fixed order (no atomics: results are bitwise
// reproducible) and fuses the vector update (residual b - A x, or
// x += omega M^{-1} r).
//
// Cells whose matrix is a scaled shared matrix (uncut cells, s K_ref; blocks
// of uncut neighbourhoods, s^{-1} inv(A_ref)) are processed as a tiled GEMM
// with the shared matrix in shared memory; cells with their own matrix (cut
// cells, irregular blocks) stream the matrix from HBM, one warp per cell,
// using the matrix symmetry so that every lane accumulates its own output
// columns without a reduction.
#include <cmath>
#include <type_traits>

#include "fcm_internal.h"

namespace fcm {

LevelGeom make_geom(int dim, int nf, int p, const int* C) {
  LevelGeom g;
  g.dim = dim;
  g.nf = nf;
  g.p = p;
  g.M = 1;
  g.nloc_s = 1;
  g.ncells = 1;
  for (int a = 0; a < 3; ++a) {
    g.C[a] = a < dim ? C[a] : 1;
    g.m[a] = a < dim ? C[a] * p + 1 : 1;
    g.M *= g.m[a];
    g.ncells *= g.C[a];
    if (a < dim) g.nloc_s *= p + 1;
  }
  g.N = g.M * nf;
  g.nloc = g.nloc_s * nf;
  return g;
}

namespace {

constexpr int kOpThreads = 256;
constexpr int kWarpsPerBlock = kOpThreads / 32;
constexpr int kTileCells = 32;
constexpr int kRowUnroll = 4;

// ---------------------------------------------------------------------------
// Stored matrices: one warp per cell.  Rows are padded to ld entries so a
// row is ld / V 16-byte vectors (V entries each).  Lanes are split into R
// row groups of ncv = ld / V lanes; lane (rg, cv) streams rows rg, rg + R, ...
// and accumulates the V output columns [cv V, cv V + V): the matrix is
// symmetric, so row s is column s and y_j += K[s][j] x_s needs no
// reduction across columns.  The R partial sums are added at the end.
template <typename TM>
struct Elem;
template <>
struct Elem<float> {
  static constexpr int V = 4;
};
template <>
struct Elem<double> {
  static constexpr int V = 2;
};
template <>
struct Elem<float2> {  // df32 pair
  static constexpr int V = 2;
};

template <typename TM>
struct Acc {
  TM v[Elem<TM>::V * 2];
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < Elem<TM>::V * 2; ++k) v[k] = 0;
  }
};
// Compensated accumulator for df32 entries: value = s + c, with the exact
// product error and the rounding error of every addition collected in c
// (TwoProduct via fma, TwoSum; Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005).
template <>
struct Acc<float2> {
  float s[4], c[4];
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] = c[k] = 0.f;
  }
};

__device__ __forceinline__ void fma_row(Acc<float>& a, int slot, const float* row, float xs) {
  float4 v = *reinterpret_cast<const float4*>(row);
  a.v[slot * 4 + 0] += v.x * xs;
  a.v[slot * 4 + 1] += v.y * xs;
  a.v[slot * 4 + 2] += v.z * xs;
  a.v[slot * 4 + 3] += v.w * xs;
}
__device__ __forceinline__ void fma_row(Acc<double>& a, int slot, const double* row, double xs) {
  double2 v = *reinterpret_cast<const double2*>(row);
  a.v[slot * 2 + 0] += v.x * xs;
  a.v[slot * 2 + 1] += v.y * xs;
}
__device__ __forceinline__ void df_term(float& s, float& c, float hi, float lo, float x) {
  float p = hi * x;
  float e = fmaf(hi, x, -p);
  float t = s + p;
  float bb = t - s;
  float err = (s - (t - bb)) + (p - bb);
  s = t;
  c += err + e + lo * x;
}
__device__ __forceinline__ void fma_row(Acc<float2>& a, int slot, const float2* row, float xs) {
  float4 v = *reinterpret_cast<const float4*>(row);  // (hi0, lo0, hi1, lo1)
  df_term(a.s[slot * 2 + 0], a.c[slot * 2 + 0], v.x, v.y, xs);
  df_term(a.s[slot * 2 + 1], a.c[slot * 2 + 1], v.z, v.w, xs);
}
__device__ __forceinline__ double acc_value(const Acc<float>& a, int k) { return a.v[k]; }
__device__ __forceinline__ double acc_value(const Acc<double>& a, int k) { return a.v[k]; }
__device__ __forceinline__ double acc_value(const Acc<float2>& a, int k) {
  return (double)a.s[k] + (double)a.c[k];
}

template <typename TV, typename TM>
__device__ void own_role(const LevelGeom& g, int ld, int n_own, const int* __restrict__ cells,
                         const TM* __restrict__ mats, const TV* __restrict__ x,
                         TV* __restrict__ Y, int vblock, int nvblocks, unsigned char* smem) {
  constexpr int V = Elem<TM>::V;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = g.nloc;
  const long long ncells = g.ncells;
  TV* xw = reinterpret_cast<TV*>(smem) + warp * 128;
  double* red = reinterpret_cast<double*>(smem + kWarpsPerBlock * 128 * sizeof(TV)) + warp * 128;
  const int ncv = ld / V;
  int R, NV;
  if (ncv <= 32) {
    R = 32 / ncv;
    NV = 1;
  } else {
    R = 1;
    NV = 2;  // ld <= 64 V
  }
  const int rg = ncv <= 32 ? lane / ncv : 0;
  const int cv = ncv <= 32 ? lane % ncv : lane;
  const bool active = rg < R;
  const bool second = NV > 1 && cv + 32 < ncv;  // second column vector of this lane
  for (int ci = vblock * kWarpsPerBlock + warp; ci < n_own; ci += nvblocks * kWarpsPerBlock) {
    const int cell = cells[ci];
    int cx, cy, cz;
    cell_coords(g, cell, cx, cy, cz);
    for (int l = lane; l < n; l += 32) xw[l] = x[cell_dof(g, cx, cy, cz, l)];
    __syncwarp();
    Acc<TM> acc;
    acc.zero();
    const TM* K = mats + (size_t)ci * n * ld;
    if (active) {
      int s = rg;
      for (; s + (kRowUnroll - 1) * R < n; s += kRowUnroll * R) {
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) {
          const int sr = s + u * R;
          const TV xs = xw[sr];
          const TM* row = K + (size_t)sr * ld;
          fma_row(acc, 0, row + cv * V, xs);
          if (second) fma_row(acc, 1, row + (cv + 32) * V, xs);
        }
      }
      for (; s < n; s += R) {
        const TV xs = xw[s];
        const TM* row = K + (size_t)s * ld;
        fma_row(acc, 0, row + cv * V, xs);
        if (second) fma_row(acc, 1, row + (cv + 32) * V, xs);
      }
    }
    if (R == 1) {
#pragma unroll
      for (int k = 0; k < 2 * V; ++k) {
        int j = (k < V ? cv * V + k : (cv + 32) * V + (k - V));
        if (k >= V && !second) break;
        if (j < n) Y[(size_t)j * ncells + cell] = (TV)acc_value(acc, k);
      }
    } else {
      if (active) {
#pragma unroll
        for (int k = 0; k < V; ++k) red[rg * ld + cv * V + k] = acc_value(acc, k);
      }
      __syncwarp();
      for (int j = lane; j < n; j += 32) {
        double t = 0.0;
        for (int r = 0; r < R; ++r) t += red[r * ld + j];
        Y[(size_t)j * ncells + cell] = (TV)t;
      }
    }
    __syncwarp();
  }
}

// Unpadded rows (ld = n not a multiple of 4): scalar loads, lane j owns the
// output columns j, j + 32, ... (row s is column s by symmetry).
__device__ void own_role_scalar(const LevelGeom& g, int n_own, const int* __restrict__ cells,
                                const double* __restrict__ mats, const double* __restrict__ x,
                                double* __restrict__ Y, int vblock, int nvblocks,
                                unsigned char* smem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = g.nloc;
  const long long ncells = g.ncells;
  double* xw = reinterpret_cast<double*>(smem) + warp * 128;
  for (int ci = vblock * kWarpsPerBlock + warp; ci < n_own; ci += nvblocks * kWarpsPerBlock) {
    const int cell = cells[ci];
    int cx, cy, cz;
    cell_coords(g, cell, cx, cy, cz);
    for (int l = lane; l < n; l += 32) xw[l] = x[cell_dof(g, cx, cy, cz, l)];
    __syncwarp();
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const double* K = mats + (size_t)ci * n * n;
    for (int s = 0; s < n; ++s) {
      const double xs = xw[s];
      const double* row = K + (size_t)s * n;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        int j = lane + 32 * k;
        if (j < n) acc[k] += row[j] * xs;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int j = lane + 32 * k;
      if (j < n) Y[(size_t)j * ncells + cell] = acc[k];
    }
    __syncwarp();
  }
}

// Shared matrices: a tile of up to 32 cells against one n x n matrix held in
// shared memory.  Thread (c = t % 32, rgroup = t / 32) computes the rows
// [rgroup R, rgroup R + R) of cell c, R = ceil(n / 8).
template <typename TV>
__device__ void tile_role(const LevelGeom& g, const int4 tile, const int* cells, const TV* scale,
                          const TV* mats, const TV* __restrict__ x, TV* __restrict__ Y,
                          TV* smem) {
  const int n = g.nloc;
  const int npad = (n + 7) & ~7;
  const int R = npad / 8;
  TV* Ks = smem;                 // n x npad
  TV* Xs = smem + n * npad;      // n x 32
  const TV* K = mats + (size_t)tile.x * n * n;
  for (int e = threadIdx.x; e < n * npad; e += blockDim.x) {
    int i = e / npad, j = e % npad;
    Ks[e] = j < n ? K[(size_t)i * n + j] : (TV)0;
  }
  const int cnt = tile.z;
  for (int e = threadIdx.x; e < n * kTileCells; e += blockDim.x) {
    int k = e / kTileCells, c = e % kTileCells;
    TV v = 0;
    if (c < cnt) {
      int cell = cells[tile.y + c];
      int cx, cy, cz;
      cell_coords(g, cell, cx, cy, cz);
      v = x[cell_dof(g, cx, cy, cz, k)];
    }
    Xs[e] = v;
  }
  __syncthreads();
  const int c = threadIdx.x % kTileCells;
  const int rg = threadIdx.x / kTileCells;
  const int i0 = rg * R;
  TV acc[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) acc[r] = 0;
  for (int k = 0; k < n; ++k) {
    TV xv = Xs[k * kTileCells + c];
    const TV* krow = Ks + k * npad + i0;  // K symmetric: K[i][k] = K[k][i]
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if (r < R) acc[r] += krow[r] * xv;
  }
  if (c < cnt) {
    const long long ncells = g.ncells;
    int cell = cells[tile.y + c];
    TV s = scale[tile.y + c];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      int i = i0 + r;
      if (r < R && i < n) Y[(size_t)i * ncells + cell] = s * acc[r];
    }
  }
  __syncthreads();
}

template <typename TV>
struct CellOpArgs {
  LevelGeom g;
  int ld;
  const TV* x;
  TV* Y;
  int n_own;
  const int* own_cells;
  const TV* own_mats;
  int n_own_x;
  const int* own_x_cells;
  const float2* own_x_mats;
  int ntiles;
  const int4* tiles;
  const int* sh_cells;
  const TV* sh_scale;
  const TV* sh_mats;
  int nb_own, nb_own_x;
};

template <typename TV>
__global__ void __launch_bounds__(kOpThreads) cell_op_kernel(CellOpArgs<TV> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int b = blockIdx.x;
  if (b < A.nb_own) {
    if constexpr (std::is_same<TV, double>::value) {
      if ((A.ld & 3) || (reinterpret_cast<uintptr_t>(A.own_mats) & 15)) {
        own_role_scalar(A.g, A.n_own, A.own_cells, A.own_mats, A.x, A.Y, b, A.nb_own, smem_raw);
        return;
      }
    }
    own_role<TV, TV>(A.g, A.ld, A.n_own, A.own_cells, A.own_mats, A.x, A.Y, b, A.nb_own,
                     smem_raw);
    return;
  }
  b -= A.nb_own;
  if (b < A.nb_own_x) {
    if constexpr (std::is_same<TV, float>::value)
      own_role<float, float2>(A.g, A.ld, A.n_own_x, A.own_x_cells, A.own_x_mats, A.x, A.Y, b,
                              A.nb_own_x, smem_raw);
    return;
  }
  b -= A.nb_own_x;
  if (b < A.ntiles)
    tile_role<TV>(A.g, A.tiles[b], A.sh_cells, A.sh_scale, A.sh_mats, A.x, A.Y,
                  reinterpret_cast<TV*>(smem_raw));
}

// ---------------------------------------------------------------------------
// DOF-centric gather of per-cell contributions (Y local-index-major).
__device__ __forceinline__ int axis_pairs(int C, int i, int& c0, int& j0, int& c1, int& j1) {
  if (i <= C) {
    if (i == 0) {
      c0 = 0;
      j0 = 0;
      return 1;
    }
    if (i == C) {
      c0 = C - 1;
      j0 = 1;
      return 1;
    }
    c0 = i - 1;
    j0 = 1;
    c1 = i;
    j1 = 0;
    return 2;
  }
  int t = i - (C + 1);
  int q = t / C;
  c0 = t - q * C;
  j0 = q + 2;
  return 1;
}

template <typename TV, int MODE>
__global__ void gather_kernel(LevelGeom g, const TV* __restrict__ Y, const TV* __restrict__ b,
                              TV* __restrict__ out, TV w) {
  const int P1 = g.p + 1;
  const long long ncells = g.ncells;
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < g.N;
       I += (long long)gridDim.x * blockDim.x) {
    const long long f = I / g.M;
    const long long r = I - f * g.M;
    const int ix = (int)(r % g.m[0]);
    const long long t = r / g.m[0];
    const int iy = (int)(t % g.m[1]);
    const int iz = (int)(t / g.m[1]);
    int cx0 = 0, jx0 = 0, cx1 = 0, jx1 = 0, cy0 = 0, jy0 = 0, cy1 = 0, jy1 = 0, cz0 = 0, jz0 = 0,
        cz1 = 0, jz1 = 0;
    const int nx = axis_pairs(g.C[0], ix, cx0, jx0, cx1, jx1);
    const int ny = g.dim > 1 ? axis_pairs(g.C[1], iy, cy0, jy0, cy1, jy1) : 1;
    const int nz = g.dim > 2 ? axis_pairs(g.C[2], iz, cz0, jz0, cz1, jz1) : 1;
    TV sum = 0;
    const int lf = (int)f * g.nloc_s;
    for (int kz = 0; kz < nz; ++kz) {
      const int cz = kz ? cz1 : cz0, jz = kz ? jz1 : jz0;
      for (int ky = 0; ky < ny; ++ky) {
        const int cy = ky ? cy1 : cy0, jy = ky ? jy1 : jy0;
        for (int kx = 0; kx < nx; ++kx) {
          const int cx = kx ? cx1 : cx0, jx = kx ? jx1 : jx0;
          const int cell = cx + g.C[0] * (cy + g.C[1] * cz);
          const int l = lf + jx + P1 * (jy + P1 * jz);
          sum += Y[(size_t)l * ncells + cell];
        }
      }
    }
    if (MODE == GATHER_SET)
      out[I] = sum;
    else if (MODE == GATHER_RESID)
      out[I] = b[I] - sum;
    else if (MODE == GATHER_ADD)
      out[I] = out[I] + w * sum;
    else
      out[I] = w * sum;
  }
}

// Canonical FP64 matrices -> padded solve layout.
__global__ void repack_kernel(int count, int n, int ld, const double* __restrict__ src,
                              const int* __restrict__ sel, int kind, void* dst) {
  long long tot = (long long)count * n * ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    int m = (int)(t / ((long long)n * ld));
    int r = (int)(t % ((long long)n * ld));
    int i = r / ld, j = r % ld;
    int sm = sel ? sel[m] : m;
    double v = j < n ? src[(size_t)sm * n * n + (size_t)i * n + j] : 0.0;
    if (kind == 0) {
      reinterpret_cast<double*>(dst)[t] = v;
    } else if (kind == 1) {
      reinterpret_cast<float*>(dst)[t] = (float)v;
    } else {
      float hi = (float)v;
      float lo = (float)(v - (double)hi);
      reinterpret_cast<float2*>(dst)[t] = make_float2(hi, lo);
    }
  }
}

// ---------------------------------------------------------------------------
// Transfers.
__device__ inline void split_index(const LevelGeom& g, long long I, long long& f, int* idx) {
  f = I / g.M;
  long long r = I - f * g.M;
  idx[0] = (int)(r % g.m[0]);
  long long t = r / g.m[0];
  idx[1] = (int)(t % g.m[1]);
  idx[2] = (int)(t / g.m[1]);
}

template <typename TV, bool PROLONG>
__global__ void p_transfer_kernel(LevelGeom gc, LevelGeom gf, const TV* in, TV* out) {
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < gc.N;
       I += (long long)gridDim.x * blockDim.x) {
    long long f;
    int idx[3];
    split_index(gc, I, f, idx);
    long long J = f * gf.M + idx[0] + (long long)gf.m[0] * (idx[1] + (long long)gf.m[1] * idx[2]);
    if (PROLONG)
      out[J] += in[I];
    else
      out[I] = in[J];
  }
}

// b_c = P^T r_f: coarse node K collects fine nodes 2K-1, 2K, 2K+1 per axis
// with weights 1/2, 1, 1/2.
template <typename TV>
__global__ void h_restrict_kernel(LevelGeom gc, LevelGeom gf, const TV* rf, TV* bc) {
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < gc.N;
       I += (long long)gridDim.x * blockDim.x) {
    long long f;
    int K[3];
    split_index(gc, I, f, K);
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      if (a < gc.dim) {
        lo[a] = 2 * K[a] - 1 < 0 ? 0 : 2 * K[a] - 1;
        hi[a] = 2 * K[a] + 1 > gf.C[a] ? gf.C[a] : 2 * K[a] + 1;
      } else {
        lo[a] = hi[a] = 0;
      }
    }
    TV sum = 0;
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          int i[3] = {x, y, z};
          TV w = 1;
          for (int a = 0; a < gc.dim; ++a)
            if (i[a] != 2 * K[a]) w *= (TV)0.5;
          sum += w * rf[f * gf.M + x + (long long)gf.m[0] * (y + (long long)gf.m[1] * z)];
        }
    bc[I] = sum;
  }
}

// x_f += P x_c: even fine node 2k takes coarse k, odd node the average of
// its two coarse neighbours.
template <typename TV>
__global__ void h_prolong_kernel(LevelGeom gc, LevelGeom gf, const TV* xc, TV* xf) {
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < gf.N;
       I += (long long)gridDim.x * blockDim.x) {
    long long f;
    int i[3];
    split_index(gf, I, f, i);
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      if (a < gf.dim) {
        c0[a] = i[a] / 2;
        c1[a] = (i[a] & 1) ? c0[a] + 1 : c0[a];
      } else {
        c0[a] = c1[a] = 0;
      }
    }
    TV sum = 0;
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) {
          int k[3] = {x, y, z};
          TV w = 1;
          for (int a = 0; a < gf.dim; ++a)
            if (c0[a] != c1[a]) w *= (TV)0.5;
          (void)k;
          sum += w * xc[f * gc.M + x + (long long)gc.m[0] * (y + (long long)gc.m[1] * z)];
        }
    xf[I] += sum;
  }
}

// x = Linv^T (Linv b), one block.
template <typename TV>
__global__ void coarse_solve_kernel(int n, const double* Linv, const TV* b, TV* x) {
  extern __shared__ double cs[];
  double* bs = cs;
  double* ys = cs + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) bs[i] = (double)b[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k <= i; ++k) s += Linv[(size_t)i * n + k] * bs[k];
    ys[i] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0;
    for (int i = j; i < n; ++i) s += Linv[(size_t)i * n + j] * ys[i];
    x[j] = (TV)s;
  }
}

// ---------------------------------------------------------------------------
// CG kernels (FP64), deterministic two-level reductions.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  s = red[32];
  __syncthreads();
  return s;
}

// Sum of kDotBlocks partials in a fixed order, done by every block.
__device__ double reduce_partials(const double* part, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) v += part[i];
  return block_sum(v, red);
}

__global__ void dot_kernel(const double* a, const double* b, long long n, double* part) {
  __shared__ double red[33];
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v += a[i] * b[i];
  double s = block_sum(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// partials of a.b and a.c
__global__ void dot2_kernel(const double* a, const double* b, const double* c, long long n,
                            double* part) {
  __shared__ double red[33];
  double v = 0.0, u = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    v += a[i] * b[i];
    u += a[i] * c[i];
  }
  double s = block_sum(v, red);
  double t = block_sum(u, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    part[kDotBlocks + blockIdx.x] = t;
  }
}

__global__ void reduce_kernel(const double* part, int count, double* out) {
  __shared__ double red[33];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += part[i];
  double s = block_sum(v, red);
  if (threadIdx.x == 0) *out = s;
}

// alpha = rz / pq; x += alpha p; r -= alpha q; partials of r.r
__global__ void cg_update_xr_kernel(double* x, double* r, const double* p, const double* q,
                                    long long n, const double* pq_part, CGScalars* sc,
                                    double* rr_part) {
  __shared__ double red[33];
  double pq = reduce_partials(pq_part, red);
  double alpha = sc->rz / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->pq = pq;
    sc->alpha = alpha;
    if (!(pq > 0.0) || !isfinite(alpha)) sc->flag = 1;
  }
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    double ri = r[i] - alpha * q[i];
    r[i] = ri;
    v += ri * ri;
  }
  double s = block_sum(v, red);
  if (threadIdx.x == 0) rr_part[blockIdx.x] = s;
}

// beta = rz_new / rz (or (rz_new - r.z_old) / rz), p = z + beta p
__global__ void cg_update_p_kernel(double* p, const double* z, long long n,
                                   const double* rz_part, int flexible, CGScalars* sc) {
  __shared__ double red[33];
  double rzn = reduce_partials(rz_part, red);
  double rzo = flexible ? reduce_partials(rz_part + kDotBlocks, red) : 0.0;
  double rz = sc->rz;
  double beta = flexible ? (rzn - rzo) / rz : rzn / rz;
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->beta = beta;
    sc->rz_new = rzn;
    if (!isfinite(beta)) sc->flag = 1;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// After the p update, rz <- rz_new (separate tiny kernel keeps the update
// kernel free of inter-block races on sc->rz).
__global__ void cg_commit_kernel(CGScalars* sc) { sc->rz = sc->rz_new; }

__global__ void cg_init_kernel(const double* z, double* p, long long n, const double* rz_part,
                               CGScalars* sc) {
  __shared__ double red[33];
  double rz = reduce_partials(rz_part, red);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rz = rz;
    sc->flag = 0;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i];
}

__global__ void d2f_kernel(const double* a, float* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f2d_kernel(const float* a, double* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
__global__ void axpby_kernel(double a, const double* x, double b, double* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
__global__ void scale_copy_kernel(const double* x, double* y, double a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
__global__ void fill_sin_kernel(double* v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = sin((double)i + 1.0);
}

inline int grid_for(long long n, int threads = 256, int cap = 8192) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace

template <typename TV>
void launch_cell_op(const LevelGeom& g, const OpData<TV>& op, const TV* x, TV* Y,
                    cudaStream_t s) {
  CellOpArgs<TV> A;
  A.g = g;
  A.ld = op.ld;
  A.x = x;
  A.Y = Y;
  A.n_own = op.own.n;
  A.own_cells = op.own.cells;
  A.own_mats = static_cast<const TV*>(op.own.mats);
  A.n_own_x = op.own_x.n;
  A.own_x_cells = op.own_x.cells;
  A.own_x_mats = static_cast<const float2*>(op.own_x.mats);
  A.ntiles = op.sh.tl.ntiles;
  A.tiles = op.sh.tl.tiles;
  A.sh_cells = op.sh.tl.cells;
  A.sh_scale = op.sh.scale;
  A.sh_mats = op.sh.mats;
  auto nb = [](int n) {
    int b = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return b > 4096 ? 4096 : b;
  };
  A.nb_own = op.own.n ? nb(op.own.n) : 0;
  A.nb_own_x = op.own_x.n ? nb(op.own_x.n) : 0;
  int grid = A.nb_own + A.nb_own_x + A.ntiles;
  if (grid == 0) return;
  int n = g.nloc, npad = (n + 7) & ~7;
  size_t sm_tile = op.sh.tl.ntiles ? ((size_t)n * npad + (size_t)n * kTileCells) * sizeof(TV) : 0;
  size_t sm_own = (size_t)kWarpsPerBlock * 128 * (sizeof(TV) + sizeof(double));
  size_t smem = sm_tile > sm_own ? sm_tile : sm_own;
  static size_t attr_set = 0;
  if (smem > 48 * 1024 && smem > attr_set) {
    cudaFuncSetAttribute(cell_op_kernel<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set = smem;
  }
  cell_op_kernel<TV><<<grid, kOpThreads, smem, s>>>(A);
}

void launch_repack(int count, int n, int ld, const double* src, const int* sel, int kind,
                   void* dst, cudaStream_t s) {
  if (count == 0) return;
  long long tot = (long long)count * n * ld;
  repack_kernel<<<grid_for(tot), 256, 0, s>>>(count, n, ld, src, sel, kind, dst);
}

template <typename TV>
void launch_gather(const LevelGeom& g, int mode, const TV* Y, const TV* b, TV* out, double w,
                   cudaStream_t s) {
  int grid = grid_for(g.N);
  TV tw = (TV)w;
  switch (mode) {
    case GATHER_SET: gather_kernel<TV, GATHER_SET><<<grid, 256, 0, s>>>(g, Y, b, out, tw); break;
    case GATHER_RESID: gather_kernel<TV, GATHER_RESID><<<grid, 256, 0, s>>>(g, Y, b, out, tw); break;
    case GATHER_ADD: gather_kernel<TV, GATHER_ADD><<<grid, 256, 0, s>>>(g, Y, b, out, tw); break;
    default: gather_kernel<TV, GATHER_SCALE><<<grid, 256, 0, s>>>(g, Y, b, out, tw); break;
  }
}

template <typename TV>
void launch_p_restrict(const LevelGeom& gc, const LevelGeom& gf, const TV* rf, TV* bc,
                       cudaStream_t s) {
  p_transfer_kernel<TV, false><<<grid_for(gc.N), 256, 0, s>>>(gc, gf, rf, bc);
}
template <typename TV>
void launch_p_prolong_add(const LevelGeom& gc, const LevelGeom& gf, const TV* xc, TV* xf,
                          cudaStream_t s) {
  p_transfer_kernel<TV, true><<<grid_for(gc.N), 256, 0, s>>>(gc, gf, xc, xf);
}
template <typename TV>
void launch_h_restrict(const LevelGeom& gc, const LevelGeom& gf, const TV* rf, TV* bc,
                       cudaStream_t s) {
  h_restrict_kernel<TV><<<grid_for(gc.N), 256, 0, s>>>(gc, gf, rf, bc);
}
template <typename TV>
void launch_h_prolong_add(const LevelGeom& gc, const LevelGeom& gf, const TV* xc, TV* xf,
                          cudaStream_t s) {
  h_prolong_kernel<TV><<<grid_for(gf.N), 256, 0, s>>>(gc, gf, xc, xf);
}
template <typename TV>
void launch_coarse_solve(int n, const double* L, const TV* b, TV* x, cudaStream_t s) {
  coarse_solve_kernel<TV><<<1, 512, 2 * n * sizeof(double), s>>>(n, L, b, x);
}

void launch_dot_partials(const double* a, const double* b, long long n, double* partials,
                         cudaStream_t s) {
  dot_kernel<<<kDotBlocks, 256, 0, s>>>(a, b, n, partials);
}
void launch_dot2_partials(const double* a, const double* b, const double* c, long long n,
                          double* partials, cudaStream_t s) {
  dot2_kernel<<<kDotBlocks, 256, 0, s>>>(a, b, c, n, partials);
}
void launch_reduce(const double* partials, int count, double* out, cudaStream_t s) {
  reduce_kernel<<<1, 256, 0, s>>>(partials, count, out);
}
void launch_cg_update_xr(double* x, double* r, const double* p, const double* q, long long n,
                         const double* pq_partials, CGScalars* sc, double* rr_partials,
                         cudaStream_t s) {
  cg_update_xr_kernel<<<kDotBlocks, 256, 0, s>>>(x, r, p, q, n, pq_partials, sc, rr_partials);
}
void launch_cg_update_p(double* p, const double* z, long long n, const double* rz_partials,
                        int flexible, CGScalars* sc, cudaStream_t s) {
  cg_update_p_kernel<<<kDotBlocks, 256, 0, s>>>(p, z, n, rz_partials, flexible, sc);
  cg_commit_kernel<<<1, 1, 0, s>>>(sc);
}
void launch_cg_init(const double* r, const double* z, long long n, const double* rz_partials,
                    double* p, CGScalars* sc, cudaStream_t s) {
  (void)r;
  cg_init_kernel<<<kDotBlocks, 256, 0, s>>>(z, p, n, rz_partials, sc);
}
void launch_copy_d2f(const double* a, float* b, long long n, cudaStream_t s) {
  d2f_kernel<<<grid_for(n), 256, 0, s>>>(a, b, n);
}
void launch_copy_f2d(const float* a, double* b, long long n, cudaStream_t s) {
  f2d_kernel<<<grid_for(n), 256, 0, s>>>(a, b, n);
}
void launch_d2f_mats(const double* a, float* b, long long n, cudaStream_t s) {
  d2f_kernel<<<grid_for(n), 256, 0, s>>>(a, b, n);
}
void launch_axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s) {
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(a, x, b, y, n);
}
void launch_scale_copy(const double* x, double* y, double a, long long n, cudaStream_t s) {
  scale_copy_kernel<<<grid_for(n), 256, 0, s>>>(x, y, a, n);
}
void launch_fill_sin(double* v, long long n, cudaStream_t s) {
  fill_sin_kernel<<<grid_for(n), 256, 0, s>>>(v, n);
}

#define FCM_INST(TV)                                                                          \
  template void launch_cell_op<TV>(const LevelGeom&, const OpData<TV>&, const TV*, TV*,        \
                                   cudaStream_t);                                              \
  template void launch_gather<TV>(const LevelGeom&, int, const TV*, const TV*, TV*, double,    \
                                  cudaStream_t);                                               \
  template void launch_p_restrict<TV>(const LevelGeom&, const LevelGeom&, const TV*, TV*,      \
                                      cudaStream_t);                                           \
  template void launch_p_prolong_add<TV>(const LevelGeom&, const LevelGeom&, const TV*, TV*,   \
                                         cudaStream_t);                                        \
  template void launch_h_restrict<TV>(const LevelGeom&, const LevelGeom&, const TV*, TV*,      \
                                      cudaStream_t);                                           \
  template void launch_h_prolong_add<TV>(const LevelGeom&, const LevelGeom&, const TV*, TV*,   \
                                         cudaStream_t);                                        \
  template void launch_coarse_solve<TV>(int, const double*, const TV*, TV*, cudaStream_t);

FCM_INST(double)
FCM_INST(float)

std::string cuda_msg(cudaError_t e) { return std::string(cudaGetErrorString(e)); }

}  // namespace fcm
