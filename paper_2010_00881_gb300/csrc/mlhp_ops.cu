// Device kernels of the multi-level hp operator (refinement by
// superposition, Sec. 2.2; the basis and leaf assembly of the paper's
// ml-hp-FCM).
//
// On an overlay mesh the matrix is summed from leaf element matrices over
// the functions supported on each leaf.  A function of ancestor level j
// restricted to a leaf of level k is a combination of the leaf's own
// (p+1)^d tensor modes with the coefficients of the Kronecker product of the
// 1D restrictions S(p, k - j, pos_a) (fcm_mlhp_restriction_1d), so the leaf
// matrix over its function list is K_L = T^T K_box T, with K_box the cell
// matrix of the leaf's box in its own modes (computed by the cell kernels of
// setup_geom.cu on the lattice of the leaf's level) and T the leaf's
// (p+1)^d x n_fun restriction matrix per field.  The load is b_L = T^T b_box.
//
// The operator is applied leaf by leaf (y_L = K_L x_L, the coefficients
// gathered through the leaf's function list) and the leaf products are
// summed per DOF through the inverse incidence lists in a fixed order, so
// results are reproducible bit for bit.
#include <cuda_runtime.h>

#include "fcm_internal.h"

namespace fcm {
namespace {

// Coefficient T[a][i] of the leaf's tensor mode a (x fastest) in the
// leaf's i-th function: the product over axes of the 1D restriction
// entries.  inc: (dk, table offsets per axis packed as tab[3], local mode per
// axis m[3]) of the incidence.
struct Inc {
  int tab[3];  // offset of the (dk, pos_a) restriction table in S (in entries)
  int m[3];    // the function's local 1D mode per axis in its ancestor
};

__device__ __forceinline__ double t_entry(const double* __restrict__ S, const Inc& in, int a,
                                          int dim, int P1) {
  double v = 1.0;
  for (int ax = 0; ax < dim; ++ax) {
    const int aa = a % P1;
    a /= P1;
    v *= S[in.tab[ax] + aa * P1 + in.m[ax]];
  }
  return v;
}

// One block per leaf: W = K_box T (field blocks), then K_L = T^T W and
// b_L = T^T b_box.  W lives in the leaf's scratch region.
__global__ void leaf_transform_kernel(int nleaf, int dim, int P1, int nf,
                                      const long long* __restrict__ off,
                                      const Inc* __restrict__ inc,
                                      const double* __restrict__ S,
                                      const double* __restrict__ Kbox,
                                      const double* __restrict__ bbox,
                                      const long long* __restrict__ koff,
                                      const long long* __restrict__ woff, double* __restrict__ W,
                                      double* __restrict__ KL, double* __restrict__ bL) {
  int ns = 1;
  for (int a = 0; a < dim; ++a) ns *= P1;
  const int n = nf * ns;
  for (int l = blockIdx.x; l < nleaf; l += gridDim.x) {
    const long long i0 = off[l];
    const int nfun = (int)(off[l + 1] - i0);
    const int nl = nf * nfun;
    const double* K = Kbox + (size_t)l * n * n;
    double* Wl = W + woff[l];
    // W[(f, a)][(f2, i2)] = sum_a2 K[(f, a)][(f2, a2)] T[a2][i2]
    for (int e = threadIdx.x; e < n * nl; e += blockDim.x) {
      const int row = e / nl, col = e % nl;
      const int f2 = col / nfun, i2 = col % nfun;
      const Inc in = inc[i0 + i2];
      double s = 0.0;
      for (int a2 = 0; a2 < ns; ++a2)
        s += K[(size_t)row * n + f2 * ns + a2] * t_entry(S, in, a2, dim, P1);
      Wl[e] = s;
    }
    __syncthreads();
    // K_L[(f, i)][(f2, i2)] = sum_a T[a][i] W[(f, a)][(f2, i2)]
    double* Kl = KL + koff[l];
    for (int e = threadIdx.x; e < nl * nl; e += blockDim.x) {
      const int r = e / nl, col = e % nl;
      const int f = r / nfun, i = r % nfun;
      const Inc in = inc[i0 + i];
      double s = 0.0;
      for (int a = 0; a < ns; ++a) s += t_entry(S, in, a, dim, P1) * Wl[(size_t)(f * ns + a) * nl + col];
      Kl[e] = s;
    }
    // b_L[(f, i)] = sum_a T[a][i] b_box[(f, a)]
    const double* bb = bbox + (size_t)l * n;
    for (int r = threadIdx.x; r < nl; r += blockDim.x) {
      const int f = r / nfun, i = r % nfun;
      const Inc in = inc[i0 + i];
      double s = 0.0;
      for (int a = 0; a < ns; ++a) s += t_entry(S, in, a, dim, P1) * bb[f * ns + a];
      bL[nf * i0 + r] = s;
    }
    __syncthreads();
  }
}

// y_L = K_L x_L, one row tile per work item: item (l, r0) computes rows
// r0 .. r0 + kLeafRows - 1 of leaf l (x_L gathered through the leaf's
// function list, field-major DOFs f M + id), so a large block spreads over
// several SMs.  K_L is symmetric, so thread r reads column r (row c,
// consecutive across threads); four partial sums over c = 0, 1, 2, 3 mod 4
// keep four loads in flight per thread and are added in a fixed order.
__global__ void __launch_bounds__(kLeafRows) leaf_apply_kernel(
    int nitem, const int2* __restrict__ items, int nf, long long M,
    const long long* __restrict__ off, const long long* __restrict__ fn,
    const long long* __restrict__ koff, const double* __restrict__ KL,
    const double* __restrict__ x, double* __restrict__ Yl) {
  extern __shared__ double xs[];
  for (int w = blockIdx.x; w < nitem; w += gridDim.x) {
    const int2 it = items[w];
    const long long i0 = off[it.x];
    const int nfun = (int)(off[it.x + 1] - i0);
    const int nl = nf * nfun;
    for (int c = threadIdx.x; c < nl; c += blockDim.x) {
      const int f = c / nfun, i = c % nfun;
      xs[c] = x[f * M + fn[i0 + i]];
    }
    __syncthreads();
    const double* Kl = KL + koff[it.x];
    const int r = it.y + (int)threadIdx.x;
    if (r < nl) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      const double* k = Kl + r;
      int c = 0;
      for (; c + 4 <= nl; c += 4) {
        s0 = fma(k[(size_t)c * nl], xs[c], s0);
        s1 = fma(k[(size_t)(c + 1) * nl], xs[c + 1], s1);
        s2 = fma(k[(size_t)(c + 2) * nl], xs[c + 2], s2);
        s3 = fma(k[(size_t)(c + 3) * nl], xs[c + 3], s3);
      }
      for (; c < nl; ++c) s0 = fma(k[(size_t)c * nl], xs[c], s0);
      Yl[nf * i0 + r] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
  }
}

// out[f M + id] = sum over the incidences of function id (in the fixed order
// of the inverse lists) of the leaf values at base + f * stride.
__global__ void leaf_gather_kernel(long long M, int nf, const long long* __restrict__ ioff,
                                   const long long* __restrict__ ibase,
                                   const int* __restrict__ istride,
                                   const double* __restrict__ Yl, double* __restrict__ out) {
  const long long N = M * nf;
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < N;
       I += (long long)gridDim.x * blockDim.x) {
    const long long f = I / M, id = I - f * M;
    double s = 0.0;
    for (long long e = ioff[id]; e < ioff[id + 1]; ++e) s += Yl[ibase[e] + f * istride[e]];
    out[I] = s;
  }
}

}  // namespace

size_t mlhp_inc_bytes() { return sizeof(Inc); }

void launch_leaf_transform(int nleaf, int dim, int P1, int nf, const long long* off,
                           const void* inc, const double* S, const double* Kbox,
                           const double* bbox, const long long* koff, const long long* woff,
                           double* W, double* KL, double* bL, cudaStream_t s) {
  if (nleaf == 0) return;
  const int grid = nleaf < 4096 ? nleaf : 4096;
  leaf_transform_kernel<<<grid, 256, 0, s>>>(nleaf, dim, P1, nf, off,
                                            static_cast<const Inc*>(inc), S, Kbox, bbox, koff,
                                            woff, W, KL, bL);
}

void launch_leaf_apply(int nitem, const int2* items, int nf, long long M, int max_nl,
                       const long long* off, const long long* fn, const long long* koff,
                       const double* KL, const double* x, double* Yl, cudaStream_t s) {
  if (nitem == 0) return;
  const int grid = nitem < 16384 ? nitem : 16384;
  leaf_apply_kernel<<<grid, kLeafRows, (size_t)max_nl * sizeof(double), s>>>(
      nitem, items, nf, M, off, fn, koff, KL, x, Yl);
}

void launch_leaf_gather(long long M, int nf, const long long* ioff, const long long* ibase,
                        const int* istride, const double* Yl, double* out, cudaStream_t s) {
  const long long N = M * nf;
  const int grid = (int)((N + 255) / 256 < 65535 ? (N + 255) / 256 : 65535);
  leaf_gather_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(M, nf, ioff, ibase, istride, Yl, out);
}

}  // namespace fcm

// ---------------------------------------------------------------------------
// hp-multigrid of overlay meshes: the level vectors are full-length
// (removed functions zero), so restriction is a mask, prolongation an add.
namespace fcm {
namespace {

enum { MV_RESID = 0, MV_AXPY = 1, MV_SCALE = 2, MV_MASK = 3, MV_ADD = 4, MV_XPBY = 5 };

// RESID: out = mask (a - b); AXPY: out += w a; SCALE: out = w a;
// MASK: out = mask a; ADD: out += a; XPBY: out = a + w out.
__global__ void mlhp_vec_kernel(long long N, int mode, const unsigned char* __restrict__ mask,
                                const double* __restrict__ a, const double* __restrict__ b,
                                double* __restrict__ out, double w) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    switch (mode) {
      case MV_RESID: out[i] = mask[i] ? a[i] - b[i] : 0.0; break;
      case MV_AXPY: out[i] += w * a[i]; break;
      case MV_SCALE: out[i] = w * a[i]; break;
      case MV_MASK: out[i] = mask[i] ? a[i] : 0.0; break;
      case MV_ADD: out[i] += a[i]; break;
      default: out[i] = a[i] + w * out[i]; break;  // MV_XPBY
    }
  }
}

}  // namespace

void launch_mlhp_vec(long long N, int mode, const unsigned char* mask, const double* a,
                     const double* b, double* out, double w, cudaStream_t s) {
  long long blocks = (N + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  mlhp_vec_kernel<<<(int)blocks, 256, 0, s>>>(N, mode, mask, a, b, out, w);
}

}  // namespace fcm

// y = A x for a CSR matrix (the Q1 levels below an overlay mesh's base
// grid and the transfers to them), one thread per row, entries summed in
// column order.
namespace fcm {
namespace {

__global__ void csr_spmv_kernel(long long rows, const long long* __restrict__ ptr,
                                const long long* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ x,
                                double* __restrict__ y) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (long long e = ptr[r]; e < ptr[r + 1]; ++e) s = fma(val[e], x[col[e]], s);
    y[r] = s;
  }
}

}  // namespace

void launch_csr_spmv(long long rows, const long long* ptr, const long long* col,
                     const double* val, const double* x, double* y, cudaStream_t s) {
  long long blocks = (rows + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  csr_spmv_kernel<<<(int)blocks, 256, 0, s>>>(rows, ptr, col, val, x, y);
}

}  // namespace fcm
