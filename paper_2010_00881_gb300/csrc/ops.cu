// Solve-path kernels of the V-cycle and of CG.
//
// Operator apply and additive Schwarz smoothing share one pattern: for every
// cell (elementwise AS blocks are cells) gather the cell's coefficients,
// multiply by a dense cell matrix (the stiffness K_c for A, the block
// inverse A_i^{-1} for M^{-1}), and write the product into a per-cell buffer
// Y[local][cell].  A second, DOF-centric pass sums the <= 2^d contributions
// of every DOF in a fixed order (no atomics: results are bitwise
// reproducible) and fuses the vector update (residual b - A x, or
// x += omega M^{-1} r).
//
// Cells whose matrix is a scaled shared matrix (uncut cells, s K_ref; blocks
// of uncut neighbourhoods, s^{-1} inv(A_ref)) are processed as a tiled GEMM
// with the shared matrix in shared memory (tile_kernel, tile_df_kernel);
// cells with their own matrix (cut cells, irregular blocks) are streamed from
// HBM through a TMA ring (stream_kernel) or, for at most 16 DOFs per cell,
// read by lane groups (small_kernel).  Every kernel uses the matrix symmetry
// (row s = column s) so that each lane accumulates its own outputs.
#include <cmath>
#include <type_traits>

#include "fcm_internal.h"
#include "tc.cuh"

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
  for (int a = 0; a < 3; ++a) g.dC[a] = make_fastdiv(g.C[a]);
  g.dm[0] = make_fastdiv(g.m[0]);
  g.dm[1] = make_fastdiv(g.m[1]);
  g.dM = make_fastdiv(g.M < 2147483647LL ? (int)g.M : 2147483647);
  return g;
}

namespace {

constexpr int kOpThreads = 256;
constexpr int kWarpsPerBlock = kOpThreads / 32;
constexpr int kTileCells = 64;
constexpr int kRowUnroll = 4;
constexpr int kOwnBlocksCap = 152 * 6;  // own-kernel blocks: several cells per warp

// Per axis the global index of mode j of cell c is c + off1(C, j): nodes
// j = 0, 1 are c and c + 1, bubble j >= 2 is (C + 1) + (j - 2) C + c.  So
// the global index of local DOF l of a cell is cell_base(cell) + tab[l],
// with tab[l] = f M + off1_x + m0 (off1_y + m1 off1_z) built once per block.
__device__ __forceinline__ int off1(int C, int j) { return j < 2 ? j : (C + 1) + (j - 2) * C; }

__device__ __forceinline__ void build_local_table(const LevelGeom& g, int* tab) {
  const int P1 = g.p + 1;
  for (int l = threadIdx.x; l < g.nloc; l += blockDim.x) {
    int f = l / g.nloc_s;
    int t = l - f * g.nloc_s;
    int jx = t % P1;
    int jy = g.dim > 1 ? (t / P1) % P1 : 0;
    int jz = g.dim > 2 ? t / (P1 * P1) : 0;
    tab[l] = f * (int)g.M + off1(g.C[0], jx) +
             g.m[0] * (off1(g.C[1], jy) + g.m[1] * off1(g.C[2], jz));
  }
}

__device__ __forceinline__ int cell_base(const LevelGeom& g, int cx, int cy, int cz) {
  return cx + g.m[0] * (cy + g.m[1] * cz);
}

// cell_base of linear cell c (x fastest), divisions by multiply-high.
__device__ __forceinline__ int cell_base_of(const LevelGeom& g, int c) {
  const int t = fdiv(g.dC[0], c);
  const int cx = c - t * g.C[0];
  const int cz = fdiv(g.dC[1], t);
  const int cy = t - cz * g.C[1];
  return cell_base(g, cx, cy, cz);
}

// Global index of the local DOF with table entry `ko` of cell (cx, cy, cz).
__device__ __forceinline__ int dof_packed(const LevelGeom& g, int cx, int cy, int cz, int ko) {
  return cell_base(g, cx, cy, cz) + ko;
}

// ---------------------------------------------------------------------------
// Lane mapping of the stored-matrix kernels (stream_kernel; own_role, the
// one-warp-per-cell fallback): rows are padded to ld entries so a row is
// ld / V 16-byte vectors (V entries each).  Lanes are split into R row groups
// of ncv = ld / V lanes; lane (rg, cv) reads rows rg, rg + R, ... and
// accumulates the V output columns [cv V, cv V + V): the matrix is
// symmetric, so row s is column s and y_j += K[s][j] x_s needs no reduction
// across columns.  The R partial sums are added at the end.
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
                         TV* __restrict__ Y, int vblock, int nvblocks, unsigned char* smem,
                         const int* tab) {
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
  const int stride = nvblocks * kWarpsPerBlock;
  int ci = vblock * kWarpsPerBlock + warp;
  // coefficients of the first cell; later cells are prefetched into
  // registers while the previous cell's matrix streams
  TV xn[4];
  if (ci < n_own) {
    int cx, cy, cz;
    cell_coords(g, cells[ci], cx, cy, cz);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int l = lane + 32 * k;
      xn[k] = l < n ? x[dof_packed(g, cx, cy, cz, tab[l])] : (TV)0;
    }
  }
  for (; ci < n_own; ci += stride) {
    const int cell = cells[ci];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int l = lane + 32 * k;
      if (l < n) xw[l] = xn[k];
    }
    __syncwarp();
    const int cnext = ci + stride;
    if (cnext < n_own) {
      int cx, cy, cz;
      cell_coords(g, cells[cnext], cx, cy, cz);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        int l = lane + 32 * k;
        if (l < n) xn[k] = x[dof_packed(g, cx, cy, cz, tab[l])];
      }
    }
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
      // with 16 < ncv < 32 column vectors the lanes past ncv hold no columns
      if (active) {
#pragma unroll
        for (int k = 0; k < 2 * V; ++k) {
          int j = (k < V ? cv * V + k : (cv + 32) * V + (k - V));
          if (k >= V && !second) break;
          if (j < n) Y[(size_t)j * ncells + cell] = (TV)acc_value(acc, k);
        }
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

// Shared matrices: a tile of up to 64 cells against one n x n matrix held in
// shared memory.  npad = next power of two >= max(16, n); thread
// (cg = t % 16, rg = t / 16) computes rows [rg RB, rg RB + RB) of the four
// cells 4 cg .. 4 cg + 3 (RB = npad / 16), so every k step reads RB matrix
// entries and 4 coefficients from shared memory for 4 RB multiply-adds.
__host__ __device__ inline int tile_npad(int n) {
  int p2 = 16;
  while (p2 < n) p2 <<= 1;
  return p2;
}

__device__ __forceinline__ uint32_t smem_addr32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization (launch_pdl) may start while its predecessor in the stream
// still runs; pdl_wait() returns once that grid has completed and its writes
// are visible (immediately for a normally launched kernel), and
// pdl_trigger() lets this kernel's dependent start early.  Only reads of the
// predecessor's results and writes to buffers it reads must follow
// pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void cp_async_4(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr32(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_8(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_addr32(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr32(dst)), "l"(src)
               : "memory");
}
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
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
  int ntiles_mma;            // tiles of <= 128 cells (tensor-core kernel, FP32)
  const int4* tiles_mma;
};

// ---------------------------------------------------------------------------
// Stored matrices streamed through shared memory by the bulk-copy (TMA)
// engine, one block per SM.  The matrices of a level's stored-matrix cells
// (up to two sets of different storage type, e.g. FP32 and df32) are cut
// into items: k whole cells when a cell fits a ring chunk, else one cell in
// cpc chunks of rc rows.  Blocks own contiguous item ranges of equal byte
// count.  A producer warp copies the block's chunks in order into a ring of
// Ring<TV>::stages 16 KB stages (full/empty mbarrier pairs); consumer warp w takes
// items w, w + kConsumers, ...: it gathers the item's coefficients with
// cp.async one item ahead, multiplies from shared memory with the
// (row group, column vector) lane mapping of own_role (row s = column s by
// symmetry) and frees the stage.  Every wait is bounded: on expiry the
// kernel records a timeout flag, and before the block exits the producer
// waits (again bounded) for the last copy issued into every stage.
// Stages per block: with FP32 vectors nine 16 KB stages still leave room for
// one tile block on the SM; with FP64 vectors (larger tiles) six.
template <typename TV>
struct Ring {
  static constexpr int stages = sizeof(TV) == 4 ? 9 : 6;
};
constexpr int kRingChunk = 16384;
constexpr int kConsumers = 8;
constexpr int kItemVals = 256;  // coefficient slots per item (cells x nloc)
constexpr long long kSpinLimit = 1LL << 26;

__device__ int g_stream_timeout = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// L2 policy for data read once per launch (the streamed matrices): evict
// first, so the vectors and per-cell products that the next kernels re-read
// stay in L2.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar, uint64_t policy) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// A parity wait names the current or the preceding phase only, so a
// consumer may wait for round r of a stage only once round r - 1 has
// completed.  Consumers take other warps' stages out of turn, so before
// the parity wait for chunk `seq` a consumer waits (bounded) until the
// producer has issued it: the producer issues a stage's round r only after
// its round r - 1 was consumed, hence completed.
__device__ __forceinline__ bool wait_issued(const volatile int* issued, long long seq) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    if (*issued > seq) {
      __threadfence_block();
      return true;
    }
    __nanosleep(32);
  }
  return false;
}

template <typename TM>
struct StreamSet {
  int n;              // cells
  const int* cells;
  const TM* mats;     // n x nloc x ld entries, cell-major
  int k;              // cells per item (> 1 only when cpc == 1)
  int cpc;            // chunks per item
  int rc;             // rows per chunk (nloc when cpc == 1)
  int items;          // ceil(n / k)
  int G;              // consumer warps per item (2: the warps split the columns)
  long long w;        // bytes per (full) item, the balancing weight
};

template <typename TV, typename TM1, typename TM2>
struct StreamArgs {
  LevelGeom g;
  int ld;
  StreamSet<TM1> s1;
  StreamSet<TM2> s2;
  const TV* x;
  TV* Y;
};

// First item of block b: byte-balanced split of the item list [set 1, set 2].
template <typename TM1, typename TM2>
__device__ __forceinline__ int block_item(const StreamSet<TM1>& a, const StreamSet<TM2>& b,
                                          int blk, int nblk) {
  const long long W1 = (long long)a.items * a.w;
  const long long W = W1 + (long long)b.items * b.w;
  const long long t = W * blk / nblk;
  long long u;
  if (t <= W1)
    u = a.w > 0 ? (t + a.w - 1) / a.w : 0;
  else
    u = a.items + (t - W1 + b.w - 1) / b.w;
  const long long T = (long long)a.items + b.items;
  return (int)(u < T ? u : T);
}

// XV: the coefficient type in shared memory (the vector type, or a float2
// (hi, lo) split of FP64 coefficients for df32 matrices).
template <typename XV, typename TM>
__device__ __forceinline__ void rows_fma(Acc<TM>& acc, const TM* K, int nrows, int ld,
                                         const XV* xs, int rg, int R, int cv, bool second) {
  constexpr int V = Elem<TM>::V;
  int r = rg;
  for (; r + 3 * R < nrows; r += 4 * R) {
    const XV x0 = xs[r], x1 = xs[r + R], x2 = xs[r + 2 * R], x3 = xs[r + 3 * R];
    const TM* row = K + (size_t)r * ld + cv * V;
    const size_t st = (size_t)R * ld;
    fma_row(acc, 0, row, x0);
    fma_row(acc, 0, row + st, x1);
    fma_row(acc, 0, row + 2 * st, x2);
    fma_row(acc, 0, row + 3 * st, x3);
    if (second) {
      fma_row(acc, 1, row + 32 * V, x0);
      fma_row(acc, 1, row + st + 32 * V, x1);
      fma_row(acc, 1, row + 2 * st + 32 * V, x2);
      fma_row(acc, 1, row + 3 * st + 32 * V, x3);
    }
  }
  for (; r < nrows; r += R) {
    const XV xv = xs[r];
    const TM* row = K + (size_t)r * ld;
    fma_row(acc, 0, row + cv * V, xv);
    if (second) fma_row(acc, 1, row + (cv + 32) * V, xv);
  }
}

// Y[jlo:jhi, cell] from the lanes' accumulators (R row groups summed in
// order; red holds R rows of the warp's W = jhi0 - jlo columns).
template <typename TV, typename TM>
__device__ __forceinline__ void store_cell(const Acc<TM>& acc, double* red, TV* Y, int cell,
                                           int n, int jlo, int W, int ncells, int R, int rg,
                                           int cv, bool active, bool second, int lane) {
  constexpr int V = Elem<TM>::V;
  if (R == 1) {
    // with 16 < ncv < 32 column vectors the lanes past ncv hold no columns
    if (active) {
#pragma unroll
      for (int k = 0; k < 2 * V; ++k) {
        const int j = (k < V ? cv * V + k : (cv + 32) * V + (k - V));
        if (k >= V && !second) break;
        if (j < n) Y[(size_t)j * ncells + cell] = (TV)acc_value(acc, k);
      }
    }
  } else {
    if (active) {
#pragma unroll
      for (int k = 0; k < V; ++k) red[rg * W + cv * V - jlo + k] = acc_value(acc, k);
    }
    __syncwarp();
    for (int j = lane; j < W && jlo + j < n; j += 32) {
      double t = 0.0;
      for (int r = 0; r < R; ++r) t += red[r * W + j];
      Y[(size_t)(jlo + j) * ncells + cell] = (TV)t;
    }
    __syncwarp();
  }
}

// Cell ids of item iu of set S: lane c < cnt holds cell c (-1 past the item).
template <typename TM>
__device__ __forceinline__ int item_ids(const StreamSet<TM>& S, int iu, int lane) {
  const int c0 = iu * S.k;
  const int cnt = min(S.k, S.n - c0);
  return lane < cnt ? S.cells[c0 + lane] : -1;
}

// Gather the coefficients of the item whose cell ids lane c holds in `ids`
// into xs (cp.async) and keep the ids in cs for the stores.
template <typename TV>
__device__ __forceinline__ void gather_ids(const LevelGeom& g, int cnt, int ids, const TV* x,
                                           TV* xs, int* cs, const int* tab, int lane) {
  const int n = g.nloc;
  if (lane < cnt) cs[lane] = ids;
  for (int c = 0; c < cnt; ++c) {
    const int cb = cell_base_of(g, __shfl_sync(0xffffffffu, ids, c));
    for (int l = lane; l < n; l += 32) {
      if constexpr (sizeof(TV) == 4)
        cp_async_4(xs + c * n + l, x + (cb + tab[l]), 4);
      else
        cp_async_8(xs + c * n + l, x + (cb + tab[l]), 8);
    }
  }
}

// Item iu of set S on warp half h of G (G = 2: the two warps of a pair take
// the column vectors [0, ceil(ncv/2)) and the rest); every warp frees each
// stage with 2 / G arrivals (empty barriers count 2).
template <typename TV, typename TM>
__device__ bool consume_item(const LevelGeom& g, int ld, const StreamSet<TM>& S, int iu,
                             int h, long long seq0, const unsigned char* ring, uint64_t* full,
                             uint64_t* empty, const volatile int* issued, const TV* xs,
                             const int* cs, double* red, TV* Y, int lane) {
  constexpr int V = Elem<TM>::V;
  constexpr int kRing = Ring<TV>::stages;
  const int n = g.nloc;
  const int ncv = ld / V;
  const int half = (ncv + 1) / 2;
  const int cv0 = S.G == 2 ? h * half : 0;
  const int ncvw = S.G == 2 ? (h == 0 ? half : ncv - half) : ncv;
  const bool any = ncvw > 0;
  const int R = !any ? 1 : (ncvw <= 32 ? 32 / ncvw : 1);
  const int rg = any && ncvw <= 32 ? lane / ncvw : 0;
  const int cv = cv0 + (any && ncvw <= 32 ? lane % ncvw : lane);
  const bool active = any && rg < R;
  const bool second = ncvw > 32 && (cv - cv0) + 32 < ncvw;
  const int jlo = cv0 * V, W = ncvw * V;
  const uint32_t arrivals = 2 / S.G;
  const int c0 = iu * S.k;
  const int cnt = min(S.k, S.n - c0);
  using XV = TV;
  const XV* xv = reinterpret_cast<const XV*>(xs);
  Acc<TM> acc;
  if (S.cpc == 1 && S.k > 1) {
    // small cells, several per chunk: lane (c, cv) multiplies all rows of
    // cell c for its column vector cv (no row groups, no reduction)
    const int slot = (int)(seq0 % kRing);
    if (!wait_issued(issued, seq0)) return false;
    if (!mbar_wait(&full[slot], (uint32_t)((seq0 / kRing) & 1))) return false;
    const TM* base = reinterpret_cast<const TM*>(ring + (size_t)slot * kRingChunk);
    const int c = lane / ncv, cvl = lane - c * ncv;
    const bool on = c < cnt;
    acc.zero();
    if (on) {
      const TM* K = base + (size_t)c * n * ld + cvl * V;
      const XV* xc = xv + c * n;
      int r = 0;
      for (; r + 3 < n; r += 4) {
        const XV x0 = xc[r], x1 = xc[r + 1], x2 = xc[r + 2], x3 = xc[r + 3];
        fma_row(acc, 0, K + (size_t)r * ld, x0);
        fma_row(acc, 0, K + (size_t)(r + 1) * ld, x1);
        fma_row(acc, 0, K + (size_t)(r + 2) * ld, x2);
        fma_row(acc, 0, K + (size_t)(r + 3) * ld, x3);
      }
      for (; r < n; ++r) fma_row(acc, 0, K + (size_t)r * ld, xc[r]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot], arrivals);
    if (on) {
      const int cell = cs[c];
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int j = cvl * V + k;
        if (j < n) Y[(size_t)j * g.ncells + cell] = (TV)acc_value(acc, k);
      }
    }
  } else if (S.cpc == 1) {
    const int slot = (int)(seq0 % kRing);
    if (!wait_issued(issued, seq0)) return false;
    if (!mbar_wait(&full[slot], (uint32_t)((seq0 / kRing) & 1))) return false;
    const TM* base = reinterpret_cast<const TM*>(ring + (size_t)slot * kRingChunk);
    bool freed = false;
    for (int c = 0; c < cnt && any; ++c) {
      acc.zero();
      if (active) rows_fma<XV, TM>(acc, base + (size_t)c * n * ld, n, ld, xv + c * n, rg, R, cv,
                                   second);
      if (c == cnt - 1) {  // the stage is free before the last cell's stores
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot], arrivals);
        freed = true;
      }
      store_cell<TV, TM>(acc, red, Y, cs[c], n, jlo, W, g.ncells, R, rg, cv, active, second,
                         lane);
    }
    if (!freed) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot], arrivals);
    }
  } else {
    acc.zero();
    for (int part = 0; part < S.cpc; ++part) {
      const long long q = seq0 + part;
      const int slot = (int)(q % kRing);
      if (!wait_issued(issued, q)) return false;
      if (!mbar_wait(&full[slot], (uint32_t)((q / kRing) & 1))) return false;
      const TM* base = reinterpret_cast<const TM*>(ring + (size_t)slot * kRingChunk);
      const int rows = min(S.rc, n - part * S.rc);
      if (active) rows_fma<XV, TM>(acc, base, rows, ld, xv + part * S.rc, rg, R, cv, second);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot], arrivals);
    }
    if (any)
      store_cell<TV, TM>(acc, red, Y, cs[0], n, jlo, W, g.ncells, R, rg, cv, active, second,
                         lane);
  }
  return true;
}

template <typename TV, typename TM1, typename TM2>
__global__ void __launch_bounds__((kConsumers + 1) * 32, 1)
    stream_kernel(StreamArgs<TV, TM1, TM2> A) {
  constexpr int kRing = Ring<TV>::stages;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int tab[128];
  __shared__ uint64_t full[kRing], empty[kRing];
  __shared__ int issued;  // chunks issued by the producer so far
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LevelGeom& g = A.g;
  build_local_table(g, tab);
  if (threadIdx.x == 0) {
    issued = 0;
    for (int k = 0; k < kRing; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 2);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const int ub = block_item(A.s1, A.s2, blockIdx.x, gridDim.x);
  const int ue = block_item(A.s1, A.s2, blockIdx.x + 1, gridDim.x);
  const int I1 = A.s1.items;
  const int a = ub > I1 ? ub : (ue < I1 ? ue : I1);  // first set-2 item of the range
  auto seq_of = [&](int u) -> long long {
    return (long long)((u < a ? u : a) - ub) * A.s1.cpc + (long long)(u > a ? u - a : 0) * A.s2.cpc;
  };
  unsigned char* ring = smem_raw;
  if (warp == kConsumers) {
    // producer
    if (lane != 0) return;
    const uint64_t policy = evict_first_policy();
    long long seq = 0;
    bool ok = true;
    for (int u = ub; u < ue && ok; ++u) {
      const bool one = u < I1;
      const int cpc = one ? A.s1.cpc : A.s2.cpc;
      for (int part = 0; part < cpc; ++part, ++seq) {
        const int slot = (int)(seq % kRing);
        if (seq >= kRing && !mbar_wait(&empty[slot], (uint32_t)(((seq / kRing) - 1) & 1))) {
          ok = false;
          break;
        }
        const void* src;
        uint32_t bytes;
        if (one) {
          const int c0 = u * A.s1.k, cnt = min(A.s1.k, A.s1.n - c0);
          src = A.s1.mats + ((size_t)c0 * g.nloc + (size_t)part * A.s1.rc) * A.ld;
          const int rows = A.s1.cpc > 1 ? min(A.s1.rc, g.nloc - part * A.s1.rc) : cnt * g.nloc;
          bytes = (uint32_t)(rows * A.ld * sizeof(TM1));
        } else {
          const int iu = u - I1;
          const int c0 = iu * A.s2.k, cnt = min(A.s2.k, A.s2.n - c0);
          src = A.s2.mats + ((size_t)c0 * g.nloc + (size_t)part * A.s2.rc) * A.ld;
          const int rows = A.s2.cpc > 1 ? min(A.s2.rc, g.nloc - part * A.s2.rc) : cnt * g.nloc;
          bytes = (uint32_t)(rows * A.ld * sizeof(TM2));
        }
        bulk_load(ring + (size_t)slot * kRingChunk, src, bytes, &full[slot], policy);
        __threadfence_block();
        *reinterpret_cast<volatile int*>(&issued) = (int)(seq + 1);
      }
    }
    if (!ok) atomicExch(&g_stream_timeout, 1);
    // the last copy issued into every stage has landed before the block's
    // shared memory goes away (consumed ones return at once)
    for (int k = 0; k < kRing; ++k) {
      if (seq > k) {
        const long long last = k + ((seq - 1 - k) / kRing) * kRing;  // last seq in stage k
        mbar_wait(&full[k], (uint32_t)((last / kRing) & 1));
      }
    }
    return;
  }
  // consumers: x comes from, and Y is read by, the preceding kernels (the
  // producer only reads the stored matrices, so it does not wait)
  pdl_wait();
  unsigned char* wbase = smem_raw + (size_t)kRing * kRingChunk +
                         (size_t)warp * (2 * kItemVals * sizeof(TV) + 128 * sizeof(double));
  TV* xb[2] = {reinterpret_cast<TV*>(wbase), reinterpret_cast<TV*>(wbase) + kItemVals};
  double* red = reinterpret_cast<double*>(wbase + 2 * kItemVals * sizeof(TV));
  __shared__ int cbuf[kConsumers][2][32];  // cell ids of the items in xb
  // this warp's items: set 1 in [ub, a), then set 2 in [a, ue); a set with
  // G = 2 gives each item to a warp pair
  const int G1 = A.s1.G, G2 = A.s2.G;
  const int f1 = ub + (G1 == 2 ? warp / 2 : warp), st1 = kConsumers / G1;
  const int f2 = a + (G2 == 2 ? warp / 2 : warp), st2 = kConsumers / G2;
  const int e2 = f2 < ue ? f2 : ue;
  auto next = [&](int v) {
    if (v >= ue) return ue;
    if (v < a) {
      v += st1;
      return v < a ? v : e2;
    }
    v += st2;
    return v < ue ? v : ue;
  };
  auto ids_of = [&](int v) {
    if (v >= ue) return -1;
    return v < I1 ? item_ids(A.s1, v, lane) : item_ids(A.s2, v - I1, lane);
  };
  auto count_of = [&](int v) {
    if (v < I1) return min(A.s1.k, A.s1.n - v * A.s1.k);
    const int iu = v - I1;
    return min(A.s2.k, A.s2.n - iu * A.s2.k);
  };
  // the ids of the item after next are loaded one iteration ahead, so no
  // dependent global load sits on the path of the item being consumed
  int u = f1 < a ? f1 : e2;
  int un = next(u);
  if (u < ue) gather_ids(g, count_of(u), ids_of(u), A.x, xb[0], cbuf[warp][0], tab, lane);
  cp_async_commit();
  int ids_n = ids_of(un);
  for (int it = 0; u < ue; ++it) {
    const int buf = it & 1;
    const int unn = next(un);
    if (un < ue) gather_ids(g, count_of(un), ids_n, A.x, xb[buf ^ 1], cbuf[warp][buf ^ 1], tab,
                            lane);
    cp_async_commit();
    ids_n = ids_of(unn);
    cp_async_wait<1>();
    __syncwarp();
    bool ok;
    if (u < I1)
      ok = consume_item<TV, TM1>(g, A.ld, A.s1, u, G1 == 2 ? (warp & 1) : 0, seq_of(u), ring,
                                 full, empty, &issued, xb[buf], cbuf[warp][buf], red, A.Y, lane);
    else
      ok = consume_item<TV, TM2>(g, A.ld, A.s2, u - I1, G2 == 2 ? (warp & 1) : 0, seq_of(u),
                                 ring, full, empty, &issued, xb[buf], cbuf[warp][buf], red, A.Y,
                                 lane);
    if (!ok) {
      if (lane == 0) atomicExch(&g_stream_timeout, 1);
      break;
    }
    __syncwarp();
    u = un;
    un = unn;
  }
  cp_async_wait<0>();
}

// Stored matrices in the vector precision (FP64 path: double; mixed: float).
template <typename TV>
__global__ void __launch_bounds__(kOpThreads) own_kernel(CellOpArgs<TV> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int tab[128];
  build_local_table(A.g, tab);
  __syncthreads();
  if constexpr (std::is_same<TV, double>::value) {
    if ((A.ld & 3) || (reinterpret_cast<uintptr_t>(A.own_mats) & 15)) {
      own_role_scalar(A.g, A.n_own, A.own_cells, A.own_mats, A.x, A.Y, blockIdx.x, gridDim.x,
                      smem_raw);
      return;
    }
  }
  own_role<TV, TV>(A.g, A.ld, A.n_own, A.own_cells, A.own_mats, A.x, A.Y, blockIdx.x, gridDim.x,
                   smem_raw, tab);
}

// Small stored matrices (n <= 16: the Q1 and p = 1 levels, 2D low degree):
// a group of L lanes per cell (N rounded up to 4, 8 or 16).  Lane j < N loads its own
// coefficient x_j and row j of the cell's matrix (row j = column j by
// symmetry; the cell's rows are one contiguous run across the group), gets
// the other coefficients by shuffles within the group and accumulates
// y_j = sum_r K[j][r] x_r in the order r = 0 .. N-1.  The row loads depend
// only on the cell's position in the list, so they overlap the cell-id ->
// coefficient chain.
template <typename TM>
struct LaneAcc;
template <>
struct LaneAcc<float> {
  float v = 0.f;
  __device__ void add(float k, float x) { v += k * x; }
  __device__ double get() const { return v; }
};
template <>
struct LaneAcc<double> {
  double v = 0.0;
  __device__ void add(double k, double x) { v += k * x; }
  __device__ double get() const { return v; }
};
template <>
struct LaneAcc<float2> {
  float s = 0.f, c = 0.f;
  __device__ void add(float2 k, float x) { df_term(s, c, k.x, k.y, x); }
  __device__ double get() const { return (double)s + (double)c; }
};

template <int N>
__host__ __device__ constexpr int lane_group() {
  return N <= 4 ? 4 : (N <= 8 ? 8 : 16);
}
// Cell sizes taken by the lane-group kernels: the Q1 and p = 1 Poisson
// levels (8 in 3D, 4 in 2D) and p = 2, 3 in 2D (9, 16).  From 24 DOFs a
// cell per warp writes its products to n scattered sectors and leaves no
// room beside it for the shared-matrix tiles: at p = 2 in 3D (n = 27) the
// stored-matrix step took 22.5 us with the tiles after it, against 16.5 us
// for the TMA ring with the tiles beside it.
__host__ __device__ constexpr bool lane_group_size(int n) {
  return n == 4 || n == 8 || n == 9 || n == 16;
}

// One cell per lane group: lane j < N multiplies row j of the cell's
// stored matrix (16-byte loads unpacked by value, so krow stays in
// registers) with the group's coefficients.
template <int N, typename TV, typename TM>
__device__ __forceinline__ void small_cell(const LevelGeom& g, const int* tab, int ci, int n,
                                           const int* __restrict__ cells,
                                           const TM* __restrict__ mats,
                                           const TV* __restrict__ x, TV* __restrict__ Y,
                                           int j) {
  constexpr int L = lane_group<N>();
  constexpr int LD = (N + 3) & ~3;
  constexpr int VE = 16 / (int)sizeof(TM);   // entries per 16-byte load
  const bool live = ci < n && j < N;
  TM krow[LD];
  if (live) {
    const float4* row = reinterpret_cast<const float4*>(mats + ((size_t)ci * N + j) * LD);
#pragma unroll
    for (int v = 0; v < LD / VE; ++v) {
      const float4 t = row[v];
      if constexpr (std::is_same<TM, float>::value) {
        krow[4 * v] = t.x;
        krow[4 * v + 1] = t.y;
        krow[4 * v + 2] = t.z;
        krow[4 * v + 3] = t.w;
      } else if constexpr (std::is_same<TM, float2>::value) {
        krow[2 * v] = make_float2(t.x, t.y);
        krow[2 * v + 1] = make_float2(t.z, t.w);
      } else {
        krow[2 * v] = __hiloint2double(__float_as_int(t.y), __float_as_int(t.x));
        krow[2 * v + 1] = __hiloint2double(__float_as_int(t.w), __float_as_int(t.z));
      }
    }
  }
  const int cell = ci < n ? cells[ci] : 0;
  const TV xj = live ? x[cell_base_of(g, cell) + tab[j]] : (TV)0;
  LaneAcc<TM> acc;
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const TV xr = __shfl_sync(0xffffffffu, xj, r, L);
    if (live) acc.add(krow[r], xr);
  }
  if (live) Y[(size_t)j * g.ncells + cell] = (TV)acc.get();
}

// Two stored sets of one level (the mixed path's FP32 and df32 matrices) in
// one launch: warps [0, W1) take set 1, the following W2 warps set 2.
template <int N, typename TV, typename TM1, typename TM2>
__global__ void __launch_bounds__(kOpThreads) small_kernel(
    LevelGeom g, int n1, const int* __restrict__ cells1, const TM1* __restrict__ mats1, int n2,
    const int* __restrict__ cells2, const TM2* __restrict__ mats2, const TV* __restrict__ x,
    TV* __restrict__ Y) {
  constexpr int L = lane_group<N>();
  constexpr int G = 32 / L;  // cells per warp
  __shared__ int tab[128];
  build_local_table(g, tab);
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int j = lane % L;
  const int W1 = (n1 + G - 1) / G, W = W1 + (n2 + G - 1) / G;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < W; w += nw) {
    if (w < W1)
      small_cell<N, TV, TM1>(g, tab, w * G + lane / L, n1, cells1, mats1, x, Y, j);
    else
      small_cell<N, TV, TM2>(g, tab, (w - W1) * G + lane / L, n2, cells2, mats2, x, Y, j);
  }
}

template <int N, typename TV, typename TM1, typename TM2>
void launch_small(const LevelGeom& g, int n1, const int* cells1, const TM1* mats1, int n2,
                  const int* cells2, const TM2* mats2, const TV* x, TV* Y, cudaStream_t s) {
  constexpr int L = lane_group<N>();
  const long long threads = ((long long)n1 + n2) * L + 2 * 32;
  int blocks = (int)((threads + kOpThreads - 1) / kOpThreads);
  if (blocks < 1) blocks = 1;
  launch_pdl(small_kernel<N, TV, TM1, TM2>, dim3(blocks), dim3(kOpThreads), 0, s, g, n1, cells1,
             mats1, n2, cells2, mats2, x, Y);
}

// Shared matrices of small cells (n in {4, 8, 9, 16}: the p = 1 level in
// 3D, p <= 3 in 2D), by the lane-group scheme of small_kernel over the
// shared-cell tiles: a tile's cells use one canonical n x n matrix (row j =
// column j) and a per-cell scale, y_c = s_c K x_c.  A block takes
// kOpThreads / L cells of one tile; lane j of a group loads column j of the
// tile's matrix (K[r][j] for r = 0 .. n-1: at each r the group reads one
// contiguous row, the same for every group, from L1) and its own
// coefficient, and gets the others by shuffles.  Compared with the tile
// kernel's gather-compute-store rounds per 64-cell tile, every cell is one
// short chain of independent loads.
template <int N, typename TV>
__global__ void __launch_bounds__(kOpThreads) small_shared_kernel(
    LevelGeom g, const int4* __restrict__ tiles, int parts, const int* __restrict__ cells,
    const TV* __restrict__ scale, const TV* __restrict__ mats, const TV* __restrict__ x,
    TV* __restrict__ Y) {
  constexpr int L = lane_group<N>();
  constexpr int CPB = kOpThreads / L;  // cells per block
  __shared__ int tab[128];
  build_local_table(g, tab);
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  const int4 t = tiles[blockIdx.x / parts];
  const int slot = (int)(blockIdx.x % parts) * CPB + (int)threadIdx.x / L;
  const int j = (int)threadIdx.x % L;
  const bool has = slot < t.z;
  const bool live = has && j < N;
  TV krow[N];
  if (live) {
    const TV* col = mats + (size_t)t.x * N * N + j;
#pragma unroll
    for (int r = 0; r < N; ++r) krow[r] = col[(size_t)r * N];
  }
  const int e = t.y + (has ? slot : 0);
  const int cell = has ? cells[e] : 0;
  const TV xj = live ? x[cell_base_of(g, cell) + tab[j]] : (TV)0;
  TV acc = (TV)0;
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const TV xr = __shfl_sync(0xffffffffu, xj, r, L);
    if (live) acc = fma(krow[r], xr, acc);
  }
  if (live) Y[(size_t)j * g.ncells + cell] = scale[e] * acc;
}

// Shared cells of small n through small_shared_kernel; false: not handled.
template <typename TV>
bool dispatch_small_shared(const CellOpArgs<TV>& A, cudaStream_t s) {
  auto go = [&](auto kernel, int L) {
    const int parts = (kTileCells * L + kOpThreads - 1) / kOpThreads;
    launch_pdl(kernel, dim3(A.ntiles * parts), dim3(kOpThreads), 0, s, A.g, A.tiles, parts,
               A.sh_cells, A.sh_scale, A.sh_mats, A.x, A.Y);
  };
  switch (A.g.nloc) {
    case 4: go(small_shared_kernel<4, TV>, 4); return true;
    case 8: go(small_shared_kernel<8, TV>, 8); return true;
    case 9: go(small_shared_kernel<9, TV>, 16); return true;
    case 16: go(small_shared_kernel<16, TV>, 16); return true;
    // from 24 DOFs a warp per cell re-reads the whole matrix per cell, and
    // the 64-cell tiles are faster (p = 2 in 3D: 8.3 against 13.6 us)
    default: return false;
  }
}

// n of lane_group_size with padded rows: lane-group kernel over the two
// stored sets (n2 = 0: one set); false: not handled here.
template <typename TV, typename TM1, typename TM2>
bool dispatch_small(const LevelGeom& g, int ld, int n1, const int* cells1, const void* mats1,
                    int n2, const int* cells2, const void* mats2, const TV* x, TV* Y,
                    cudaStream_t s) {
  const int n = g.nloc;
  if (ld != padded_ld(n) || (reinterpret_cast<uintptr_t>(mats1) & 15) ||
      (reinterpret_cast<uintptr_t>(mats2) & 15))
    return false;
  const TM1* m1 = static_cast<const TM1*>(mats1);
  const TM2* m2 = static_cast<const TM2*>(mats2);
  switch (n) {
#define FCM_SMALL_CASE(NN)                                                                  \
  case NN:                                                                                  \
    launch_small<NN, TV, TM1, TM2>(g, n1, cells1, m1, n2, cells2, m2, x, Y, s);             \
    return true;
    FCM_SMALL_CASE(4)
    FCM_SMALL_CASE(8)
    FCM_SMALL_CASE(9)
    FCM_SMALL_CASE(16)
#undef FCM_SMALL_CASE
    default: return false;
  }
}

// Stored df32 islands of the mixed path (float vectors).
__global__ void __launch_bounds__(kOpThreads) own_x_kernel(CellOpArgs<float> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int tab[128];
  build_local_table(A.g, tab);
  __syncthreads();
  own_role<float, float2>(A.g, A.ld, A.n_own_x, A.own_x_cells, A.own_x_mats, A.x, A.Y,
                          blockIdx.x, gridDim.x, smem_raw, tab);
}

// Shared matrices: persistent blocks walk the tile list (tiles of up to 64
// cells against one n x n matrix, K symmetric so row k = column k).  The
// matrix stays in shared memory while consecutive tiles use it; matrix and
// coefficients arrive by cp.async (the next tile's coefficients are
// gathered into the second buffer while the current tile is multiplied).
// npad = next power of two >= max(16, n); thread (cg = t % 16, rg = t / 16)
// computes rows [rg RB, rg RB + RB) of the cells 4 cg .. 4 cg + 3.  The
// products are staged through shared memory so each row of Y is written as
// one coalesced run over the tile's cells.
template <typename TV, int RB, int NB>
__global__ void __launch_bounds__(kOpThreads) tile_kernel(CellOpArgs<TV> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int tab[128];
  __shared__ int ccell[2][2][kTileCells];  // cell (-1: empty slot), cell_base
  __shared__ TV cscale[2][kTileCells];
  constexpr int npad = 16 * RB;
  constexpr int lgp = RB == 1 ? 4 : RB == 2 ? 5 : RB == 4 ? 6 : 7;
  constexpr int V16 = 16 / (int)sizeof(TV);  // entries per 16-byte copy
  const LevelGeom& g = A.g;
  const int n = g.nloc;
  TV* Ks = reinterpret_cast<TV*>(smem_raw);
  TV* Xb[2] = {Ks + n * npad, Ks + n * npad + (NB == 2 ? n * kTileCells : 0)};
  build_local_table(g, tab);
  const int T = A.ntiles;
  int t = blockIdx.x;
  if (t >= T) return;
  auto coords = [&](int tt, int buf) {
    if (threadIdx.x < kTileCells) {
      const int4 tl = A.tiles[tt];
      const int c = threadIdx.x;
      const int cell = c < tl.z ? A.sh_cells[tl.y + c] : 0;
      int cx, cy, cz;
      cell_coords(g, cell, cx, cy, cz);
      ccell[buf][0][c] = c < tl.z ? cell : -1;
      ccell[buf][1][c] = cell_base(g, cx, cy, cz);
      cscale[buf][c] = c < tl.z ? A.sh_scale[tl.y + c] : (TV)0;
    }
  };
  auto gather = [&](int buf) {
    TV* X = Xb[buf];
    for (int e = threadIdx.x; e < n * kTileCells; e += blockDim.x) {
      const int k = e >> 6, c = e & (kTileCells - 1);
      const bool live = ccell[buf][0][c] >= 0;
      const TV* src = live ? A.x + (ccell[buf][1][c] + tab[k]) : A.x;
      if constexpr (sizeof(TV) == 4)
        cp_async_4(X + e, src, live ? 4 : 0);
      else
        cp_async_8(X + e, src, live ? 8 : 0);
    }
    cp_async_commit();
  };
  // rows of K into Ks[k][0 .. n); 16-byte copies when rows start aligned
  auto load_matrix = [&](int m) {
    const TV* K = A.sh_mats + (size_t)m * n * n;
    if (n % V16 == 0 && (reinterpret_cast<uintptr_t>(A.sh_mats) & 15) == 0) {
      const int nv = n / V16;
      for (int e = threadIdx.x; e < n * nv; e += blockDim.x) {
        const int k = e / nv, v = e - k * nv;
        cp_async_16(Ks + k * npad + v * V16, K + (size_t)k * n + v * V16);
      }
    } else {
      for (int e = threadIdx.x; e < n * npad; e += blockDim.x) {
        const int i = e >> lgp, j = e & (npad - 1);
        const TV* src = j < n ? K + (size_t)i * n + j : K;
        if constexpr (sizeof(TV) == 4)
          cp_async_4(Ks + e, src, j < n ? 4 : 0);
        else
          cp_async_8(Ks + e, src, j < n ? 8 : 0);
      }
    }
    cp_async_commit();
  };
  if (NB == 2) {
    coords(t, 0);
    __syncthreads();
    gather(0);
  }
  int cur_mat = -1;
  const int cg = threadIdx.x & 15;
  const int rg = threadIdx.x >> 4;
  const int i0 = rg * RB;
  const long long ncells = g.ncells;
  for (int it = 0; t < T; t += gridDim.x, ++it) {
    const int buf = NB == 2 ? (it & 1) : 0;
    const int tn = t + gridDim.x;
    const int4 tile = A.tiles[t];
    if (NB == 2) {
      if (tn < T) coords(tn, buf ^ 1);
    } else {
      coords(t, 0);
    }
    if (tile.x != cur_mat) {
      load_matrix(tile.x);
      cur_mat = tile.x;
    }
    __syncthreads();
    // groups complete in issue order: [this tile's X] [K] [next tile's X]
    if (NB == 2) {
      if (tn < T) {
        gather(buf ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    } else {
      gather(0);
      cp_async_wait<0>();
    }
    __syncthreads();
    TV* Xs = Xb[buf];
    TV acc[RB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0;
    if (i0 < n) {
#pragma unroll 2
      for (int k = 0; k < n; ++k) {
        TV xv[4];
        const TV* xr = Xs + k * kTileCells + 4 * cg;
        TV kv[RB];
        const TV* kr = Ks + k * npad + i0;
        if constexpr (std::is_same<TV, float>::value) {
          float4 q = *reinterpret_cast<const float4*>(xr);
          xv[0] = q.x; xv[1] = q.y; xv[2] = q.z; xv[3] = q.w;
          if constexpr (RB >= 4) {
#pragma unroll
            for (int r4 = 0; r4 < RB / 4; ++r4) {
              float4 u = *reinterpret_cast<const float4*>(kr + 4 * r4);
              kv[4 * r4] = u.x; kv[4 * r4 + 1] = u.y; kv[4 * r4 + 2] = u.z; kv[4 * r4 + 3] = u.w;
            }
          } else {
#pragma unroll
            for (int r = 0; r < RB; ++r) kv[r] = kr[r];
          }
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) xv[c] = xr[c];
#pragma unroll
          for (int r = 0; r < RB; ++r) kv[r] = kr[r];
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] += kv[r] * xv[c];
      }
    }
    __syncthreads();  // every thread is done reading Xs
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = i0 + r;
      if (i < n) {
#pragma unroll
        for (int c = 0; c < 4; ++c) Xs[i * kTileCells + 4 * cg + c] = acc[r][c];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * kTileCells; e += blockDim.x) {
      const int i = e >> 6, c = e & (kTileCells - 1);
      const int cell = ccell[buf][0][c];
      if (cell >= 0) A.Y[(size_t)i * ncells + cell] = cscale[buf][c] * Xs[e];
    }
    __syncthreads();
  }
}

// Shared operator matrix of uncut Poisson cells by sum factorisation (FP64).
// The uncut cell matrix is the Kronecker sum K = sum_a (x)_b F_ab with
// F_ab = K1_a (1D stiffness) if a == b and M1_b (1D mass) otherwise (Sec.
// 2.1; tensor-product basis, x fastest).  Applied to a cell's coefficient
// tensor X (P^D values) as 1D contractions along the axes, reusing partial
// products: D = 3: U = M_x X, V = K_x X; W = M_y V + K_y U, T = M_y U;
// Y = M_z W + K_z T (7 P^4 multiply-adds instead of P^6); D = 2: U = M_x X,
// V = K_x X; Y = M_y V + K_y U.  GB300's FP64 rate is 1/64 of its FP32 rate
// and this product is bound by it, so fewer FMAs is what counts.  A block
// takes 64-cell tiles in batches of CT cells staged in shared memory (three
// buffers of CT x P^D values, rows padded by one to spread banks); each
// thread contracts whole lines (P values along one axis) from registers.
template <int P, int D, int CT>
__global__ void __launch_bounds__(kOpThreads) kron_tile_kernel(CellOpArgs<double> A,
                                                               const double* __restrict__ kron) {
  constexpr int NL = D == 3 ? P * P * P : P * P;  // values per cell
  constexpr int LD = NL + 1;                      // padded row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int tab[128];
  __shared__ double F[D][2][P * P];               // [axis][K1, M1]
  __shared__ int ccell[CT], cbase[CT];
  __shared__ double cscale[CT];
  double* B0 = reinterpret_cast<double*>(smem_raw);
  double* B1 = B0 + CT * LD;
  double* B2 = B1 + CT * LD;
  const LevelGeom& g = A.g;
  build_local_table(g, tab);
  for (int e = threadIdx.x; e < D * 2 * P * P; e += blockDim.x) (&F[0][0][0])[e] = kron[e];
  const long long ncells = g.ncells;
  // contraction of one line: out[i] = sum_j Mat[i][j] in[j]
  auto line = [&](const double* M, const double* in, double* out) {
#pragma unroll
    for (int i = 0; i < P; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < P; ++j) s = fma(M[i * P + j], in[j], s);
      out[i] = s;
    }
  };
  for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
    const int4 tile = A.tiles[t];
    for (int c0 = 0; c0 < tile.z; c0 += CT) {
      const int cnt = min(CT, tile.z - c0);
      __syncthreads();
      if (threadIdx.x < CT) {
        const int c = threadIdx.x;
        const bool live = c < cnt;
        const int cell = live ? A.sh_cells[tile.y + c0 + c] : 0;
        int cx, cy, cz;
        cell_coords(g, cell, cx, cy, cz);
        ccell[c] = live ? cell : -1;
        cbase[c] = cell_base(g, cx, cy, cz);
        cscale[c] = live ? A.sh_scale[tile.y + c0 + c] : 0.0;
      }
      __syncthreads();
      // gather X (consecutive threads: consecutive cells of one local DOF)
      for (int e = threadIdx.x; e < NL * CT; e += blockDim.x) {
        const int l = e / CT, c = e - l * CT;
        B0[c * LD + l] = ccell[c] >= 0 ? __ldg(A.x + cbase[c] + tab[l]) : 0.0;
      }
      __syncthreads();
      // pass 1, along x (stride 1): U = M_x X -> B1, V = K_x X -> B2
      for (int e = threadIdx.x; e < CT * (NL / P); e += blockDim.x) {
        const int c = e / (NL / P), r = e - c * (NL / P);
        const double* in = B0 + c * LD + r * P;
        double v[P], o[P];
#pragma unroll
        for (int j = 0; j < P; ++j) v[j] = in[j];
        line(F[0][1], v, o);
#pragma unroll
        for (int j = 0; j < P; ++j) B1[c * LD + r * P + j] = o[j];
        line(F[0][0], v, o);
#pragma unroll
        for (int j = 0; j < P; ++j) B2[c * LD + r * P + j] = o[j];
      }
      __syncthreads();
      // pass 2, along y (stride P): lines (c, x, z)
      for (int e = threadIdx.x; e < CT * (NL / P); e += blockDim.x) {
        const int c = e / (NL / P), r = e - c * (NL / P);
        const int ix = r % P, iz = r / P;
        const int base = c * LD + ix + iz * P * P;
        double u[P], v[P], o1[P], o2[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
          u[j] = B1[base + j * P];
          v[j] = B2[base + j * P];
        }
        line(F[1][1], v, o1);   // M_y V
        line(F[1][0], u, o2);   // K_y U
#pragma unroll
        for (int j = 0; j < P; ++j) B0[base + j * P] = o1[j] + o2[j];   // Y (2D) or W (3D)
        if constexpr (D == 3) {
          line(F[1][1], u, o1);                                            // T = M_y U
#pragma unroll
          for (int j = 0; j < P; ++j) B2[base + j * P] = o1[j];
        }
      }
      __syncthreads();
      const double* Yb = B0;
      if constexpr (D == 3) {
        // pass 3, along z (stride P^2): Y = M_z W + K_z T -> B1
        for (int e = threadIdx.x; e < CT * P * P; e += blockDim.x) {
          const int c = e / (P * P), r = e - c * (P * P);
          const int base = c * LD + r;
          double w[P], tt[P], o1[P], o2[P];
#pragma unroll
          for (int j = 0; j < P; ++j) {
            w[j] = B0[base + j * P * P];
            tt[j] = B2[base + j * P * P];
          }
          line(F[2][1], w, o1);
          line(F[2][0], tt, o2);
#pragma unroll
          for (int j = 0; j < P; ++j) B1[base + j * P * P] = o1[j] + o2[j];
        }
        __syncthreads();
        Yb = B1;
      }
      for (int e = threadIdx.x; e < NL * CT; e += blockDim.x) {
        const int l = e / CT, c = e - l * CT;
        if (ccell[c] >= 0) A.Y[(size_t)l * ncells + ccell[c]] = cscale[c] * Yb[c * LD + l];
      }
    }
  }
}

// Shared matrices on the tensor cores (FP32 vectors).  For a tile of up to
// 128 cells that share one matrix K (n x n, symmetric), the products are
// D = X K with X the tile's gathered coefficients, one row per cell: one
// M = 128, N = NP (n padded to a multiple of 16) GEMM with reduction length
// KD (n padded to a multiple of 8).  Both operands are split into TF32
// parts, v = hi + lo with hi = tf32(v) and lo = v - hi (exact in FP32), and
// D = Xh Kh + Xh Kl + Xl Kh accumulates in FP32 in tensor memory (3xTF32,
// about FP32 accuracy; the dropped Xl Kl term is below 2^-22 |X||K|).  K's
// parts, split once at setup into the operand layout, arrive by one bulk
// copy and stay in shared memory while consecutive tiles use the same
// matrix; X is gathered through the per-cell DOF table in chunks of KC
// values of K (KC < KD when the block must fit beside a stored-matrix
// streaming block on the SM).  Thread 0 issues the MMAs and commits them to
// an mbarrier; every wait is bounded (on expiry the timeout flag is set and
// the block stops after a second bounded wait for what is in flight).
// Epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (one cell
// per lane) and writes s_c D[c][j] to Y[j][cell], consecutive cells to
// consecutive addresses.
constexpr int kMmaCells = 128;
constexpr int kMmaMinN = 48;  // DOFs per cell from which the tensor-core tiles are used
constexpr int kMmaMinForked = 24;  // the same beside a streaming block
constexpr uint32_t kMmaWaitLimit = 1u << 24;

template <int RV>
__global__ void __launch_bounds__(kMmaCells) tc_tile_kernel(CellOpArgs<float> A,
                                                             const float* __restrict__ mma_b,
                                                             int KD, int NP, int KC,
                                                             uint32_t ncols) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ int tab[128];
  __shared__ int ccell[kMmaCells];
  __shared__ int cbase[kMmaCells];
  __shared__ float cscale[kMmaCells];
  __shared__ __align__(8) uint64_t mbar;   // MMA completion
  __shared__ __align__(8) uint64_t bbar;   // B operand arrival
  __shared__ uint32_t tslot;
  const LevelGeom& g = A.g;
  const int n = g.nloc;
  const uint32_t bbytes = (uint32_t)NP * KD * 4;
  char* Bh = reinterpret_cast<char*>(smem_raw);
  char* Bl = Bh + bbytes;
  char* Ah = Bl + bbytes;
  char* Al = Ah + (size_t)kMmaCells * KC * 4;
  build_local_table(g, tab);
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_init(&bbar, 1);
  }
  if (threadIdx.x < 32) tc::tmem_alloc(&tslot, ncols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t idesc = tc::make_idesc_tf32(kMmaCells, NP);
  const uint32_t sboA = (uint32_t)(KC / 4) * 128u, sboB = (uint32_t)(KD / 4) * 128u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ncells = g.ncells;
  int cur_mat = -1;
  uint32_t phase = 0, bphase = 0;
  bool b_pending = false, failed = false;
  for (int t = blockIdx.x; t < A.ntiles_mma && !failed; t += gridDim.x) {
    const int4 tile = A.tiles_mma[t];
    if (tile.x != cur_mat) {
      // the MMAs of the previous tile have completed (waited below)
      if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         tc::smem_u32(&bbar)),
                     "r"(2u * bbytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(tc::smem_u32(Bh)),
            "l"(mma_b + (size_t)tile.x * 2 * NP * KD), "r"(2u * bbytes),
            "r"(tc::smem_u32(&bbar))
            : "memory");
      }
      b_pending = true;
      cur_mat = tile.x;
    }
    if (threadIdx.x < kMmaCells) {
      const int c = threadIdx.x;
      const bool live = c < tile.z;
      const int cell = live ? A.sh_cells[tile.y + c] : 0;
      int cx, cy, cz;
      cell_coords(g, cell, cx, cy, cz);
      ccell[c] = live ? cell : -1;
      cbase[c] = cell_base(g, cx, cy, cz);
      cscale[c] = live ? A.sh_scale[tile.y + c] : 0.f;
    }
    __syncthreads();
    // thread c gathers cell c's values in passes of RV (all loads of a pass
    // issued before the first is used: one round of loads per pass), then
    // feeds the pass's chunks of KC (a divisor of RV) to the tensor cores,
    // splitting and storing kc / 4 16-byte vectors per chunk
    const int c_me = threadIdx.x;
    const bool live = ccell[c_me] >= 0;
    const float* xb = A.x + cbase[c_me];
    float v[RV];
    for (int k0 = 0; k0 < KD; k0 += KC) {
      const int kc = KD - k0 < KC ? KD - k0 : KC;
      const int p0 = k0 - k0 % RV;  // first k of this pass
      if (k0 == p0) {
#pragma unroll
        for (int i = 0; i < RV; ++i) {
          const int k = p0 + i;
          v[i] = (live && k < n) ? __ldg(xb + tab[k]) : 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < RV / 4; ++i) {
        const int kk = 4 * i - (k0 - p0);  // position within the chunk
        if (kk >= 0 && kk < kc) {
          float4 hv, lv;
          hv.x = tc::to_tf32(v[4 * i + 0]); lv.x = v[4 * i + 0] - hv.x;
          hv.y = tc::to_tf32(v[4 * i + 1]); lv.y = v[4 * i + 1] - hv.y;
          hv.z = tc::to_tf32(v[4 * i + 2]); lv.z = v[4 * i + 2] - hv.z;
          hv.w = tc::to_tf32(v[4 * i + 3]); lv.w = v[4 * i + 3] - hv.w;
          const uint32_t off = tc::kmajor_offset(c_me, kk, KC);
          *reinterpret_cast<float4*>(Ah + off) = hv;
          *reinterpret_cast<float4*>(Al + off) = lv;
        }
      }
      tc::fence_proxy_async();
      __syncthreads();
      bool ok = true;
      if (threadIdx.x == 0) {
        if (b_pending) {
          ok = tc::mbar_wait(&bbar, bphase, kMmaWaitLimit);
          if (ok) {
            bphase ^= 1u;
            b_pending = false;
          }
        }
        if (ok) {
          tc::fence_after_sync();
          const uint32_t ah0 = tc::smem_u32(Ah), al0 = tc::smem_u32(Al);
          const uint32_t bh0 = tc::smem_u32(Bh) + (uint32_t)(k0 / 8) * 256u;
          const uint32_t bl0 = tc::smem_u32(Bl) + (uint32_t)(k0 / 8) * 256u;
          for (int s = 0; s < kc / 8; ++s) {
            const uint64_t ah = tc::make_sdesc(ah0 + 256u * s, 128u, sboA);
            const uint64_t al = tc::make_sdesc(al0 + 256u * s, 128u, sboA);
            const uint64_t bh = tc::make_sdesc(bh0 + 256u * s, 128u, sboB);
            const uint64_t bl = tc::make_sdesc(bl0 + 256u * s, 128u, sboB);
            tc::mma_tf32(tmem, ah, bh, idesc, (k0 > 0 || s > 0) ? 1u : 0u);
            tc::mma_tf32(tmem, ah, bl, idesc, 1u);
            tc::mma_tf32(tmem, al, bh, idesc, 1u);
          }
          tc::commit(&mbar);
        }
      }
      // the chunk's MMAs must finish before its operands are overwritten
      if (__syncthreads_or(!ok)) {
        // B never arrived: no MMA was issued; let the copy land (bounded)
        if (threadIdx.x == 0) {
          atomicExch(&g_stream_timeout, 1);
          tc::mbar_wait(&bbar, bphase, kMmaWaitLimit);
        }
        failed = true;
        break;
      }
      ok = tc::mbar_wait(&mbar, phase, kMmaWaitLimit);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicExch(&g_stream_timeout, 1);
        tc::mbar_wait(&mbar, phase, kMmaWaitLimit);
        failed = true;
        break;
      }
      phase ^= 1u;
    }
    if (failed) break;
    tc::fence_after_sync();
    {
      const int lg = warp & 3;
      const int c = 32 * lg + lane;
      const int cell = ccell[c];
      const float sc = cscale[c];
      for (int ch = 0; 16 * ch < n; ++ch) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + 16u * ch, v);
        if (cell >= 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int j = 16 * ch + i;
            if (j < n) A.Y[(size_t)j * ncells + cell] = sc * v[i];
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_free(tmem, ncols);
}

// Operand layout of launch_mma_operands: thread e of matrix m handles one
// (j, k) entry, reading K[k][j] (K symmetric; rows contiguous across threads).
__global__ void mma_operands_kernel(int n, int KD, int NP, int nmats, const float* mats,
                                    float* out) {
  const long long per = (long long)NP * KD;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * nmats;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e / per);
    const int r = (int)(e - (long long)m * per);
    const int k = r / NP, j = r - k * NP;
    const float v = (j < n && k < n) ? mats[(size_t)m * n * n + (size_t)k * n + j] : 0.f;
    const float hi = tc::to_tf32(v);
    const uint32_t off = tc::kmajor_offset(j, k, KD) / 4;
    out[(size_t)m * 2 * per + off] = hi;
    out[(size_t)m * 2 * per + per + off] = v - hi;
  }
}



// ---------------------------------------------------------------------------
// DOF-centric gather of per-cell contributions (Y local-index-major).
__device__ __forceinline__ int axis_pairs(int C, const FastDiv& dC, int i, int& c0, int& j0,
                                          int& c1, int& j1) {
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
  const int t = i - (C + 1);
  const int q = fdiv(dC, t);
  c0 = t - q * C;
  j0 = q + 2;
  return 1;
}

// Contributions of DOF I = f M + ix + m0 (iy + m1 iz): the (up to 2 per
// axis) cells that share the DOF and its local index in each are found per
// axis (divisions by multiply-high); all (up to 8) values are loaded before
// any is added, absent ones read as 0.
template <typename TV>
__device__ __forceinline__ void gather_load(const LevelGeom& g, const TV* __restrict__ Y, int I,
                                            bool live, TV v[8]) {
  const int P1 = g.p + 1;
  const int ncells = g.ncells;
  const int f = g.nf > 1 ? fdiv(g.dM, I) : 0;
  const int r = I - f * (int)g.M;
  const int t = fdiv(g.dm[0], r);
  const int ix = r - t * g.m[0];
  const int iz = fdiv(g.dm[1], t);
  const int iy = t - iz * g.m[1];
  int cx0 = 0, jx0 = 0, cx1 = 0, jx1 = 0;
  int cy0 = 0, jy0 = 0, cy1 = 0, jy1 = 0, cz0 = 0, jz0 = 0, cz1 = 0, jz1 = 0;
  const int nx = axis_pairs(g.C[0], g.dC[0], ix, cx0, jx0, cx1, jx1);
  const int ny = g.dim > 1 ? axis_pairs(g.C[1], g.dC[1], iy, cy0, jy0, cy1, jy1) : 1;
  const int nz = g.dim > 2 ? axis_pairs(g.C[2], g.dC[2], iz, cz0, jz0, cz1, jz1) : 1;
  const int lf = f * g.nloc_s;
#pragma unroll
  for (int kz = 0; kz < 2; ++kz) {
    const int cz = kz ? cz1 : cz0, jz = kz ? jz1 : jz0;
#pragma unroll
    for (int ky = 0; ky < 2; ++ky) {
      const int cy = ky ? cy1 : cy0, jy = ky ? jy1 : jy0;
      const bool on = live && kz < nz && ky < ny;
      const int cyz = g.C[0] * (cy + g.C[1] * cz);
      const int lyz = lf + P1 * (jy + P1 * jz);
      const TV* Yb = Y + (size_t)lyz * ncells + cyz;
      v[4 * kz + 2 * ky] = on ? Yb[(size_t)jx0 * ncells + cx0] : (TV)0;
      v[4 * kz + 2 * ky + 1] = (on && nx > 1) ? Yb[(size_t)jx1 * ncells + cx1] : (TV)0;
    }
  }
}

template <typename TV, int MODE>
__device__ __forceinline__ void gather_store(const TV v[8], const TV* __restrict__ b,
                                             TV* __restrict__ out, TV w, int I) {
  TV sum = 0;  // fixed order: cells (z, y, x)
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += v[k];
  if (MODE == GATHER_SET)
    out[I] = sum;
  else if (MODE == GATHER_RESID)
    out[I] = b[I] - sum;
  else if (MODE == GATHER_ADD)
    out[I] = out[I] + w * sum;
  else
    out[I] = w * sum;
}

// kGatherDofs DOFs per thread (I, I + stride, ...), all their loads in
// flight before any sum.
constexpr int kGatherDofs = 1;
template <typename TV, int MODE>
__global__ void __launch_bounds__(256) gather_kernel(LevelGeom g, const TV* __restrict__ Y,
                                                     const TV* __restrict__ b,
                                                     TV* __restrict__ out, TV w) {
  pdl_wait();
  pdl_trigger();  // the next cell kernel may start streaming its matrices
  const int N = (int)g.N;
  const int stride = gridDim.x * blockDim.x;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += kGatherDofs * stride) {
    TV v[kGatherDofs][8];
#pragma unroll
    for (int u = 0; u < kGatherDofs; ++u) {
      const int Iu = I + u * stride;
      gather_load<TV>(g, Y, Iu < N ? Iu : I, Iu < N, v[u]);
    }
#pragma unroll
    for (int u = 0; u < kGatherDofs; ++u) {
      const int Iu = I + u * stride;
      if (Iu < N) gather_store<TV, MODE>(v[u], b, out, w, Iu);
    }
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
  pdl_wait();
  pdl_trigger();
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
  pdl_wait();
  pdl_trigger();
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
    // the up to 3 x 3 x 3 fine nodes, loaded together, summed in (z, y, x)
    // order; absent ones are skipped
    TV v[3][3][3];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int x = lo[0] + dx, y = lo[1] + dy, z = lo[2] + dz;
          const bool on = x <= hi[0] && y <= hi[1] && z <= hi[2];
          v[dz][dy][dx] =
              on ? rf[f * gf.M + x + (long long)gf.m[0] * (y + (long long)gf.m[1] * z)] : (TV)0;
        }
    TV sum = 0;
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int x = lo[0] + dx, y = lo[1] + dy, z = lo[2] + dz;
          if (x > hi[0] || y > hi[1] || z > hi[2]) continue;
          const int i[3] = {x, y, z};
          TV w = 1;
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (a < gc.dim && i[a] != 2 * K[a]) w *= (TV)0.5;
          sum += w * v[dz][dy][dx];
        }
    bc[I] = sum;
  }
}

// x_f += P x_c: even fine node 2k takes coarse k, odd node the average of
// its two coarse neighbours.
template <typename TV>
__global__ void h_prolong_kernel(LevelGeom gc, LevelGeom gf, const TV* xc, TV* xf) {
  pdl_wait();
  pdl_trigger();
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
// x = Linv^T (Linv b), one block.  One warp per row of each triangular
// product; lanes stride the row and a butterfly adds their partial sums
// (fixed order: deterministic).  A warp takes kCoarseRows rows at a time and
// each lane loads all its entries of a 128-column slab before the FMAs, so
// the row loads overlap instead of following one another.
constexpr int kCoarseRows = 4;
template <typename TV>
__global__ void __launch_bounds__(1024) coarse_solve_kernel(int n, const double* __restrict__ Linv,
                                                           const TV* b, TV* x) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double cs[];
  double* bs = cs;
  double* ys = cs + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) bs[i] = (double)b[i];
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i0 = w; i0 < n; i0 += nw * kCoarseRows) {
    double s[kCoarseRows] = {};
    for (int kb = 0; kb < n; kb += 128) {
      double v[kCoarseRows][4];
#pragma unroll
      for (int r = 0; r < kCoarseRows; ++r)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int i = i0 + r * nw, k = kb + l + 32 * m;
          v[r][m] = (i < n && k <= i) ? Linv[(size_t)i * n + k] : 0.0;
        }
#pragma unroll
      for (int r = 0; r < kCoarseRows; ++r)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int i = i0 + r * nw, k = kb + l + 32 * m;
          if (i < n && k <= i) s[r] += v[r][m] * bs[k];
        }
    }
#pragma unroll
    for (int r = 0; r < kCoarseRows; ++r) {
      double t = s[r];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      const int i = i0 + r * nw;
      if (l == 0 && i < n) ys[i] = t;
    }
  }
  __syncthreads();
  for (int j0 = w; j0 < n; j0 += nw * kCoarseRows) {
    double s[kCoarseRows] = {};
    for (int ib = 0; ib < n; ib += 128) {
      double v[kCoarseRows][4];
#pragma unroll
      for (int r = 0; r < kCoarseRows; ++r)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int j = j0 + r * nw, i = j + ib + l + 32 * m;
          v[r][m] = (j < n && i < n) ? Linv[(size_t)i * n + j] : 0.0;
        }
#pragma unroll
      for (int r = 0; r < kCoarseRows; ++r)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int j = j0 + r * nw, i = j + ib + l + 32 * m;
          if (j < n && i < n) s[r] += v[r][m] * ys[i];
        }
    }
#pragma unroll
    for (int r = 0; r < kCoarseRows; ++r) {
      double t = s[r];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      const int j = j0 + r * nw;
      if (l == 0 && j < n) x[j] = (TV)t;
    }
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

template <typename TV, int RB>
void launch_tile(const CellOpArgs<TV>& A, size_t /*sm_one_buffer*/, cudaStream_t s,
                 bool one_per_sm) {
  // FP32: two coefficient buffers; as many persistent blocks as shared
  // memory keeps resident (at most four per SM), each walking several tiles
  // so the next tile's gather overlaps the current product.  FP64: the
  // product is FMA-bound on this GPU; one tile per block, single buffer.
  constexpr int NB = sizeof(TV) == 8 ? 1 : 2;
  const int n = A.g.nloc;
  const size_t smem = ((size_t)n * 16 * RB + (size_t)NB * n * kTileCells) * sizeof(TV);
  // set once, to the largest tile this instantiation can need (n <= 16 RB),
  // so concurrent callers never lower it under each other's launches
  static const bool attr = [] {
    const size_t mx =
        ((size_t)16 * RB * 16 * RB + (size_t)NB * 16 * RB * kTileCells) * sizeof(TV);
    cudaFuncSetAttribute(tile_kernel<TV, RB, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)mx);
    // full shared-memory carveout, so tile blocks fit beside stream blocks
    cudaFuncSetAttribute(tile_kernel<TV, RB, NB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         100);
    return true;
  }();
  (void)attr;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = (int)((200 * 1024) / (smem + 4096));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  int grid = one_per_sm ? sms : (NB == 2 ? sms * per_sm : A.ntiles);
  if (grid > A.ntiles) grid = A.ntiles;
  tile_kernel<TV, RB, NB><<<grid, kOpThreads, smem, s>>>(A);
}

// Tensor-core tiles (FP32 vectors, n <= 128): K padded to KD (multiple of
// 8) and N to NP (multiple of 16); the gathered coefficients come in chunks
// of KC values, as many as `budget` bytes of shared memory hold beside K's
// two parts (KC = 0: they do not fit).
int mma_rv(int n) {  // values per thread and gather pass: KD up to a power of two, <= 64
  int rv = 8;
  while (rv < mma_kd(n) && rv < 64) rv <<= 1;
  return rv;
}
int mma_chunk(int n, size_t budget) {
  const size_t bsz = (size_t)2 * mma_np(n) * mma_kd(n) * 4;
  if (bsz >= budget) return 0;
  const int fit = (int)((budget - bsz) / (2 * kMmaCells * 4));
  // a power of two (a divisor of the pass length), at most one pass
  int KC = 8;
  if (fit < 8) return 0;
  while (2 * KC <= fit && 2 * KC <= mma_rv(n)) KC <<= 1;
  return KC;
}

// Persistent blocks of 128 threads (one warp per SM sub-partition, so that a
// block fits beside a streaming block's nine warps in every sub-partition's
// register file) walk the 128-cell tile list; as many per SM as shared
// memory admits (one when they run beside stored-matrix streaming blocks),
// at most eight, and never more than the SM's 512 tensor-memory columns hold
// (ncols each).  The kernel's attributes are set by
// prepare_kernels(), outside any stream capture.
void launch_tc_tile(const CellOpArgs<float>& A, const float* mma_b, int KC, bool one_per_sm,
                    cudaStream_t s) {
  const int n = A.g.nloc;
  const int KD = mma_kd(n), NP = mma_np(n);
  uint32_t ncols = 32;
  while ((int)ncols < NP) ncols <<= 1;
  const size_t smem = (size_t)2 * NP * KD * 4 + (size_t)2 * kMmaCells * KC * 4;
  int dev = 0, sms = 148, smem_sm = 228 * 1024;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int per_sm = (int)((size_t)smem_sm / (smem + 3 * 1024));
  if (per_sm > 8) per_sm = 8;
  if (per_sm > (int)(512 / ncols)) per_sm = (int)(512 / ncols);
  if (per_sm < 1 || one_per_sm) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > A.ntiles_mma) grid = A.ntiles_mma;
  switch (mma_rv(n)) {
    case 8: tc_tile_kernel<8><<<grid, kMmaCells, smem, s>>>(A, mma_b, KD, NP, KC, ncols); break;
    case 16: tc_tile_kernel<16><<<grid, kMmaCells, smem, s>>>(A, mma_b, KD, NP, KC, ncols); break;
    case 32: tc_tile_kernel<32><<<grid, kMmaCells, smem, s>>>(A, mma_b, KD, NP, KC, ncols); break;
    default: tc_tile_kernel<64><<<grid, kMmaCells, smem, s>>>(A, mma_b, KD, NP, KC, ncols); break;
  }
}

// Sum-factorised shared tiles (FP64, Poisson): P = p + 1, D = dim; batches
// of 32 cells (16 when a cell has more than 64 DOFs), three shared-memory
// buffers of about 50 KB together, so a block fits beside a streaming block.
inline int kron_ct(int nl) { return nl <= 64 ? 32 : 16; }
inline size_t kron_smem(int nl) { return (size_t)3 * kron_ct(nl) * (nl + 1) * sizeof(double); }

template <int P, int D>
void launch_kron_p(const CellOpArgs<double>& A, const double* kron, int grid, cudaStream_t s) {
  constexpr int NL = D == 3 ? P * P * P : P * P;
  constexpr int CT = NL <= 64 ? 32 : 16;
  kron_tile_kernel<P, D, CT><<<grid, kOpThreads, kron_smem(NL), s>>>(A, kron);
}

bool kron_supported(int dim, int p) {
  return (dim == 3 && p >= 1 && p <= 4) || (dim == 2 && p >= 1 && p <= 8);
}

void launch_kron_tile(const CellOpArgs<double>& A, const double* kron, bool one_per_sm,
                      cudaStream_t s) {
  const int nl = A.g.nloc;
  int dev = 0, sms = 148, smem_sm = 228 * 1024;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int per_sm = (int)((size_t)smem_sm / (kron_smem(nl) + 4 * 1024));
  if (per_sm > 4) per_sm = 4;
  if (per_sm < 1 || one_per_sm) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > A.ntiles) grid = A.ntiles;
  const int P = A.g.p + 1;
  if (A.g.dim == 3) {
    switch (P) {
      case 2: launch_kron_p<2, 3>(A, kron, grid, s); break;
      case 3: launch_kron_p<3, 3>(A, kron, grid, s); break;
      case 4: launch_kron_p<4, 3>(A, kron, grid, s); break;
      default: launch_kron_p<5, 3>(A, kron, grid, s); break;
    }
  } else {
    switch (P) {
      case 2: launch_kron_p<2, 2>(A, kron, grid, s); break;
      case 3: launch_kron_p<3, 2>(A, kron, grid, s); break;
      case 4: launch_kron_p<4, 2>(A, kron, grid, s); break;
      case 5: launch_kron_p<5, 2>(A, kron, grid, s); break;
      case 6: launch_kron_p<6, 2>(A, kron, grid, s); break;
      case 7: launch_kron_p<7, 2>(A, kron, grid, s); break;
      case 8: launch_kron_p<8, 2>(A, kron, grid, s); break;
      default: launch_kron_p<9, 2>(A, kron, grid, s); break;
    }
  }
}

void launch_mma_operands(int n, int nmats, const float* mats, float* out, cudaStream_t s) {
  if (nmats == 0) return;
  const long long tot = (long long)nmats * mma_np(n) * mma_kd(n);
  mma_operands_kernel<<<grid_for(tot), 256, 0, s>>>(n, mma_kd(n), mma_np(n), nmats, mats, out);
}

template <typename K>
cudaError_t prepare_one(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

cudaError_t prepare_kernels() {
  // dynamic shared memory up to the opt-in limit minus the static part
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = prepare_one(tc_tile_kernel<8>, optin);
  if (e == cudaSuccess) e = prepare_one(tc_tile_kernel<16>, optin);
  if (e == cudaSuccess) e = prepare_one(tc_tile_kernel<32>, optin);
  if (e == cudaSuccess) e = prepare_one(tc_tile_kernel<64>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<2, 3, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<3, 3, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<4, 3, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<5, 3, 16>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<2, 2, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<3, 2, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<4, 2, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<5, 2, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<6, 2, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<7, 2, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<8, 2, 32>, optin);
  if (e == cudaSuccess) e = prepare_one(kron_tile_kernel<9, 2, 16>, optin);
  return e;
}

// Items of a stored-matrix set: k whole cells per ring chunk when a cell
// fits (at most kItemVals coefficients per item), else one cell in cpc
// chunks of rc rows (as many rows as fit; the last chunk holds the rest).
template <typename TM>
StreamSet<TM> make_stream_set(int n, const int* cells, const void* mats, int nloc, int ld) {
  StreamSet<TM> S;
  S.n = n;
  S.cells = cells;
  S.mats = static_cast<const TM*>(mats);
  const size_t row = (size_t)ld * sizeof(TM), cb = row * nloc;
  if (cb <= (size_t)kRingChunk) {
    int k = (int)(kRingChunk / cb);
    if (k > kItemVals / nloc) k = kItemVals / nloc;
    // several cells per item are taken side by side, a lane per (cell,
    // column vector): at most 32 such pairs
    const int ncv = ld / Elem<TM>::V;
    if (k > 1 && k * ncv > 32) k = 32 / ncv > 1 ? 32 / ncv : 1;
    S.k = k < 1 ? 1 : k;
    S.cpc = 1;
    S.rc = nloc;
  } else {
    const int rc = (int)(kRingChunk / row);  // full chunks; the last one is shorter
    S.k = 1;
    S.rc = rc;
    S.cpc = (nloc + rc - 1) / rc;
  }
  S.items = n > 0 ? (n + S.k - 1) / S.k : 0;
  S.G = S.cpc > 1 ? 2 : 1;
  S.w = (long long)S.k * (long long)cb;
  return S;
}

// Launch with programmatic stream serialization (see pdl_wait).
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename TV, typename TM1, typename TM2>
void launch_stream(const StreamArgs<TV, TM1, TM2>& S, cudaStream_t s) {
  const size_t smem = (size_t)Ring<TV>::stages * kRingChunk +
                      (size_t)kConsumers * (2 * kItemVals * sizeof(TV) + 128 * sizeof(double));
  static const bool attr = [smem] {
    cudaFuncSetAttribute(stream_kernel<TV, TM1, TM2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    // full shared-memory carveout, so tile blocks fit beside stream blocks
    cudaFuncSetAttribute(stream_kernel<TV, TM1, TM2>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return true;
  }();
  (void)attr;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int items = S.s1.items + S.s2.items;
  const int grid = items < sms ? items : sms;
  if (grid > 0)
    launch_pdl(stream_kernel<TV, TM1, TM2>, dim3(grid), dim3((kConsumers + 1) * 32), smem, s, S);
}

template <typename TV>
void launch_cell_op(const LevelGeom& g, const OpData<TV>& op, const TV* x, TV* Y,
                    cudaStream_t s, const SideStream* side) {
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
  A.ntiles_mma = op.sh.tl.ntiles_mma;
  A.tiles_mma = op.sh.tl.tiles_mma;
  auto nb = [](int n) {
    int b = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return b > kOwnBlocksCap ? kOwnBlocksCap : b;
  };
  A.nb_own = op.own.n ? nb(op.own.n) : 0;
  A.nb_own_x = op.own_x.n ? nb(op.own_x.n) : 0;
  int n = g.nloc;
  const size_t sm_own = (size_t)kWarpsPerBlock * 128 * (sizeof(TV) + sizeof(double));
  const int ld = op.ld;
  // With stored-matrix work to overlap them with, the tiles go on the side
  // stream, forked before and issued after the stored-matrix kernels (whose
  // persistent blocks then hold one slot per SM), as one persistent block
  // per SM that fits beside them.  Tiles too large to fit beside a stream
  // block (n > 64 at FP32, n > 32 at FP64) run after it with their usual
  // grid instead.
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const bool al = (ld & 3) == 0 && al16(op.own.mats) && al16(op.own_x.mats);
  const bool small = lane_group_size(n) && ld == padded_ld(n) && al;
  // FP32 vectors: the shared-matrix products run on the tensor cores
  // (tc_tile_kernel) from kMmaMinN DOFs per cell up, with the operand chunk
  // KC sized so that one block fits beside a streaming block when they run
  // side by side.  Below that the product is a few hundred FMAs per cell and
  // the CUDA-core tiles finish sooner than the tensor-core kernel's fixed
  // latency (tensor-memory allocation, MMA commit and wait: about 5 us).
  const bool mma_ok = std::is_same<TV, float>::value && A.ntiles_mma > 0 && n <= 128 &&
                      op.sh.mma_b != nullptr;
  bool mma = mma_ok && n >= kMmaMinN;
  int KC = mma ? mma_chunk(n, 200 * 1024) : 0;
  const bool stored = A.nb_own || A.nb_own_x;
  // beside a streaming block the CUDA-core tiles get one block per SM; from
  // kMmaMinForked DOFs per cell the tensor-core tiles finish sooner there
  // (the operator at p = 2 in 3D: 14.4 against 16.5 us per step; not the
  // smoother's many shared inverses, 22.5 against 20.5 us, see below)
  if (!mma && mma_ok && n >= kMmaMinForked && side && side->s2 && stored &&
      !lane_group_size(n))
    mma = true;
  // shared memory left on an SM beside one streaming block (12 KB: static
  // shared memory of both kernels and the per-block reservations)
  size_t left = 0;
  if (side && side->s2 && stored && !small) {
    const size_t stream_smem =
        (size_t)Ring<TV>::stages * kRingChunk +
        (size_t)kConsumers * (2 * kItemVals * sizeof(TV) + 128 * sizeof(double));
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    left = (size_t)per_sm > stream_smem + 12 * 1024 ? (size_t)per_sm - stream_smem - 12 * 1024 : 0;
  }
  if (mma && op.sh.mma_only_alone && side && side->s2 && stored) {
    const int npad = tile_npad(n);
    const size_t cc_smem = ((size_t)n * npad + 2 * (size_t)n * kTileCells) * sizeof(TV);
    if (small || cc_smem <= left) mma = false;  // CUDA-core tiles run beside the stream
  }
  bool fork = side && side->s2 && (mma ? A.ntiles_mma : A.ntiles) && stored;
  if (fork && !small) {
    if (mma) {
      const int kc = mma_chunk(n, left);
      fork = kc >= 8;
      if (fork) KC = kc;
    } else if (op.sh.kron) {
      fork = kron_smem(n) <= left;
    } else {
      const int npad = tile_npad(n);
      const size_t tile_smem =
          ((size_t)n * npad + (sizeof(TV) == 4 ? 2 : 1) * (size_t)n * kTileCells) * sizeof(TV);
      fork = tile_smem <= left;
    }
  }
  if (fork) cudaEventRecord(side->fork, s);
  if (A.nb_own || A.nb_own_x) {
    if (small) {
      if constexpr (std::is_same<TV, float>::value)
        dispatch_small<float, float, float2>(g, ld, op.own.n, op.own.cells, op.own.mats,
                                             op.own_x.n, op.own_x.cells, op.own_x.mats, x, Y, s);
      else
        dispatch_small<double, double, double>(g, ld, op.own.n, op.own.cells, op.own.mats, 0,
                                               nullptr, nullptr, x, Y, s);
    } else if (al && n <= 128) {
      if constexpr (std::is_same<TV, float>::value) {
        StreamArgs<float, float, float2> S{
            g, ld, make_stream_set<float>(op.own.n, op.own.cells, op.own.mats, n, ld),
            make_stream_set<float2>(op.own_x.n, op.own_x.cells, op.own_x.mats, n, ld), x, Y};
        launch_stream(S, s);
      } else {
        StreamArgs<double, double, double> S{
            g, ld, make_stream_set<double>(op.own.n, op.own.cells, op.own.mats, n, ld),
            make_stream_set<double>(0, nullptr, nullptr, n, ld), x, Y};
        launch_stream(S, s);
      }
    } else {
      if (A.nb_own) own_kernel<TV><<<A.nb_own, kOpThreads, sm_own, s>>>(A);
      if constexpr (std::is_same<TV, float>::value) {
        if (A.nb_own_x) {
          const size_t smx = (size_t)kWarpsPerBlock * 128 * (sizeof(float) + sizeof(double));
          own_x_kernel<<<A.nb_own_x, kOpThreads, smx, s>>>(A);
        }
      }
    }
  }
  if (mma) {
    cudaStream_t st = s;
    if (fork) {
      cudaStreamWaitEvent(side->s2, side->fork, 0);
      st = side->s2;
    }
    if constexpr (std::is_same<TV, float>::value)
      launch_tc_tile(A, op.sh.mma_b, KC, fork && !small, st);
    if (fork) {
      cudaEventRecord(side->join, side->s2);
      cudaStreamWaitEvent(s, side->join, 0);
    }
  } else if (A.ntiles) {
    cudaStream_t st = s;
    if (fork) {
      cudaStreamWaitEvent(side->s2, side->fork, 0);
      st = side->s2;
    }
    const int npad = tile_npad(n);
    size_t sm_tile = ((size_t)n * npad + (size_t)n * kTileCells) * sizeof(TV);
    // one block per SM only beside stream blocks; the small-cell kernels
    // leave the SMs' shared memory free
    const bool one = fork && !small;
    bool done = false;
    if constexpr (std::is_same<TV, double>::value) {
      if (op.sh.kron) {
        launch_kron_tile(A, op.sh.kron, one, st);
        done = true;
      }
    }
    if (!done) done = dispatch_small_shared<TV>(A, st);
    if (done) {
      if (fork) {
        cudaEventRecord(side->join, side->s2);
        cudaStreamWaitEvent(s, side->join, 0);
      }
      return;
    }
    switch (npad / 16) {
      case 1: launch_tile<TV, 1>(A, sm_tile, st, one); break;
      case 2: launch_tile<TV, 2>(A, sm_tile, st, one); break;
      case 4: launch_tile<TV, 4>(A, sm_tile, st, one); break;
      default: launch_tile<TV, 8>(A, sm_tile, st, one); break;
    }
    if (fork) {
      cudaEventRecord(side->join, side->s2);
      cudaStreamWaitEvent(s, side->join, 0);
    }
  }
}

// Diagonal of a level operator, cell by cell: Y[l][c] = (K_c)_{ll}, the
// stored matrix's entry for stored cells and s_c (K_ref)_{ll} for cells that
// share a matrix; the DOF gather then sums the diagonals of the cells at a
// DOF (Jacobi smoother, Sec. 4.1).
__global__ void cell_diag_kernel(LevelGeom g, int ld, int n_own, const int* own_cells,
                                 const double* own_mats, int n_sh, const int* sh_cells,
                                 const int* sh_mat, const double* sh_scale,
                                 const double* sh_mats, double* Y) {
  const int n = g.nloc;
  const long long ncells = g.ncells;
  const long long tot = (long long)(n_own + n_sh) * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), l = (int)(e - (long long)i * n);
    if (i < n_own) {
      Y[(size_t)l * ncells + own_cells[i]] = own_mats[((size_t)i * n + l) * ld + l];
    } else {
      const int j = i - n_own;
      Y[(size_t)l * ncells + sh_cells[j]] =
          sh_scale[j] * sh_mats[((size_t)sh_mat[j] * n + l) * n + l];
    }
  }
}

// x = w dinv r (init) or x += w dinv r.
template <typename TV>
__global__ void jacobi_kernel(long long N, const TV* dinv, const TV* r, TV* x, TV w, int init) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const TV z = w * (dinv[i] * r[i]);
    x[i] = init ? z : x[i] + z;
  }
}

void launch_cell_diag(const LevelGeom& g, const OpData<double>& op, const int* sh_mat,
                      double* Y, cudaStream_t s) {
  const long long tot = (long long)(op.own.n + op.sh.tl.ncells) * g.nloc;
  if (tot == 0) return;
  cell_diag_kernel<<<grid_for(tot), 256, 0, s>>>(
      g, op.ld, op.own.n, op.own.cells, static_cast<const double*>(op.own.mats),
      op.sh.tl.ncells, op.sh.tl.cells, sh_mat, op.sh.scale, op.sh.mats, Y);
}

template <typename TV>
void launch_jacobi(long long N, const TV* dinv, const TV* r, TV* x, double w, bool init,
                   cudaStream_t s) {
  jacobi_kernel<TV><<<grid_for(N), 256, 0, s>>>(N, dinv, r, x, (TV)w, init ? 1 : 0);
}
template void launch_jacobi<double>(long long, const double*, const double*, double*, double,
                                    bool, cudaStream_t);
template void launch_jacobi<float>(long long, const float*, const float*, float*, double, bool,
                                   cudaStream_t);

// Trunk space (the paper's 3D elements, Sec. 4.3): of the (p+1)^d tensor
// modes of a cell, the trunk space of degree q keeps those whose bubble
// degrees (local mode j >= 2 has degree j) sum to at most q.  The library
// keeps the tensor layout and removes the other modes from the system: their
// rows and columns of every cell matrix and block inverse are zero and their
// load entries zero, so iterates and corrections stay zero on them.
__device__ __forceinline__ bool trunk_masked_local(int l, int dim, int nloc_s, int P, int q) {
  int s = l % nloc_s, sum = 0;
  for (int a = 0; a < dim; ++a) {
    const int j = s % P;
    s /= P;
    if (j >= 2) sum += j;
  }
  return sum > q;
}

__global__ void trunk_mask_mats_kernel(long long count, int dim, int nf, int p, int q, int unit,
                                       double* mats) {
  const int P = p + 1;
  int nloc_s = 1;
  for (int a = 0; a < dim; ++a) nloc_s *= P;
  const int n = nf * nloc_s;
  const long long tot = count * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int rc = (int)(e % ((long long)n * n));
    const int r = rc / n, c = rc - r * n;
    const bool mr = trunk_masked_local(r, dim, nloc_s, P, q);
    const bool mc = trunk_masked_local(c, dim, nloc_s, P, q);
    if (mr || mc) mats[e] = (unit && r == c) ? 1.0 : 0.0;
  }
}

__global__ void trunk_mask_vec_kernel(LevelGeom g, int q, double* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    long long t = i % g.M;
    int sum = 0;
    for (int a = 0; a < g.dim; ++a) {
      const int ia = (int)(t % g.m[a]);
      t /= g.m[a];
      if (ia > g.C[a]) sum += 2 + (ia - g.C[a] - 1) / g.C[a];
    }
    if (sum > q) v[i] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Node-centric level operations (p = 1 and Q1 levels, n = nf 2^d).  On
// these levels a cell product and its DOF gather are each a few
// microseconds of dependent loads on small vectors; one pass per half step
// halves the launches.  A group of 2^d lanes serves one DOF (field f, node
// i): lane s takes the cell on side s of the node, multiplies row
// l = f 2^d + k of the cell's matrix (k: the node's corner in the cell; row
// l = column l by symmetry) with the cell's coefficients read from x (a
// df32 row with compensated accumulation, a shared row scaled by the
// cell's factor), and the group sums the 2^d products in lane order.  The
// arithmetic per product and the summation order across cells are those of
// the cell kernels and the gather.
template <int D, int NF, typename TV, typename TM2, int MODE>
__global__ void __launch_bounds__(256) node_kernel(LevelGeom g, NodeSet<TV> op,
                                                   const TV* __restrict__ x,
                                                   const TV* __restrict__ b,
                                                   TV* __restrict__ out, TV w) {
  constexpr int NS = 1 << D;  // nodes per cell = lanes per DOF
  constexpr int N = NF * NS;  // DOFs per cell
  pdl_wait();
  pdl_trigger();
  const int Ntot = (int)g.N, M = (int)g.M;
  const int m0 = g.m[0], m1 = D == 3 ? g.m[1] : 1;
  const TV* __restrict__ A1 = static_cast<const TV*>(op.m1);
  const TM2* __restrict__ A2 = static_cast<const TM2*>(op.m2);
  const int lane = threadIdx.x & 31;
  const int sl = lane % NS;  // the cell side: bit a set = the cell above the node on axis a
  const int stride = (gridDim.x * blockDim.x) / NS;
  // every lane of a warp runs the same number of iterations (the shuffles)
  const int total = (Ntot + stride - 1) / stride;
  int I = (blockIdx.x * blockDim.x + threadIdx.x) / NS;
  for (int it = 0; it < total; ++it, I += stride) {
    TV part = (TV)0;
    if (I < Ntot) {
      const int f = I / M;
      const int r = I - f * M;
      const int ix = r % m0;
      const int iy = D == 3 ? (r / m0) % m1 : r / m0;
      const int iz = D == 3 ? r / (m0 * m1) : 0;
      const int sx = sl & 1, sy = (sl >> 1) & 1, sz = D == 3 ? (sl >> 2) & 1 : 0;
      const int cx = ix - 1 + sx, cy = iy - 1 + sy, cz = D == 3 ? iz - 1 + sz : 0;
      if (cx >= 0 && cx < g.C[0] && cy >= 0 && cy < g.C[1] && cz >= 0 && cz < g.C[2]) {
        const int k = (1 - sx) + 2 * (1 - sy) + 4 * (D == 3 ? 1 - sz : 0);
        const int l = f * NS + k;
        const int cell = cx + g.C[0] * (cy + g.C[1] * cz);
        const int nb = cx + m0 * (cy + m1 * cz);  // the cell's first node
        TV xc[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
          const int f2 = q / NS, k2 = q % NS;
          xc[q] = x[f2 * M + nb + (k2 & 1) + m0 * ((k2 >> 1) & 1) + m0 * m1 * (k2 >> 2)];
        }
        const int cd = op.code[cell];
        if (cd >= 0) {
          const TV* row = A1 + ((size_t)cd * N + l) * op.ld;
#pragma unroll
          for (int q = 0; q < N; ++q) part = fma(row[q], xc[q], part);
        } else if (cd <= -2) {
          if constexpr (std::is_same<TM2, float2>::value) {
            const float2* row = A2 + ((size_t)(-cd - 2) * N + l) * op.ld;
            float s0 = 0.f, c0 = 0.f;
#pragma unroll
            for (int q = 0; q < N; ++q) df_term(s0, c0, row[q].x, row[q].y, xc[q]);
            part = (TV)((double)s0 + (double)c0);
          }
        } else {
          const TV* row = op.sh + ((size_t)op.mat[cell] * N + l) * N;
          TV t = (TV)0;
#pragma unroll
          for (int q = 0; q < N; ++q) t = fma(row[q], xc[q], t);
          part = op.scale[cell] * t;
        }
      }
    }
    // fixed-order sum over the group's lanes
    TV y = __shfl_sync(0xffffffffu, part, 0, NS);
#pragma unroll
    for (int q = 1; q < NS; ++q) y += __shfl_sync(0xffffffffu, part, q, NS);
    if (I < Ntot && sl == 0) {
      if (MODE == GATHER_SET)
        out[I] = y;
      else if (MODE == GATHER_RESID)
        out[I] = b[I] - y;
      else if (MODE == GATHER_ADD)
        out[I] = out[I] + w * y;
      else
        out[I] = w * y;
    }
  }
}

template <int D, int NF, typename TV>
void launch_node_dn(const LevelGeom& g, const NodeSet<TV>& op, const TV* x, const TV* b, TV* out,
                    TV w, int mode, cudaStream_t s) {
  using TM2 = typename std::conditional<std::is_same<TV, float>::value, float2, double>::type;
  const long long threads = g.N * (1LL << D);
  const int grid = (int)((threads + 255) / 256);
  switch (mode) {
    case GATHER_SET:
      launch_pdl(node_kernel<D, NF, TV, TM2, GATHER_SET>, dim3(grid), dim3(256), 0, s, g, op, x, b,
                 out, w);
      break;
    case GATHER_RESID:
      launch_pdl(node_kernel<D, NF, TV, TM2, GATHER_RESID>, dim3(grid), dim3(256), 0, s, g, op, x,
                 b, out, w);
      break;
    case GATHER_ADD:
      launch_pdl(node_kernel<D, NF, TV, TM2, GATHER_ADD>, dim3(grid), dim3(256), 0, s, g, op, x, b,
                 out, w);
      break;
    default:
      launch_pdl(node_kernel<D, NF, TV, TM2, GATHER_SCALE>, dim3(grid), dim3(256), 0, s, g, op, x,
                 b, out, w);
      break;
  }
}

template <typename TV>
void launch_node(const LevelGeom& g, const NodeSet<TV>& op, const TV* x, const TV* b, TV* out,
                 double w, int mode, cudaStream_t s) {
  const TV tw = (TV)w;
  if (g.dim == 3 && g.nf == 1) launch_node_dn<3, 1, TV>(g, op, x, b, out, tw, mode, s);
  else if (g.dim == 3 && g.nf == 3) launch_node_dn<3, 3, TV>(g, op, x, b, out, tw, mode, s);
  else if (g.dim == 2 && g.nf == 1) launch_node_dn<2, 1, TV>(g, op, x, b, out, tw, mode, s);
  else launch_node_dn<2, 2, TV>(g, op, x, b, out, tw, mode, s);
}
template void launch_node<float>(const LevelGeom&, const NodeSet<float>&, const float*,
                                 const float*, float*, double, int, cudaStream_t);
template void launch_node<double>(const LevelGeom&, const NodeSet<double>&, const double*,
                                  const double*, double*, double, int, cudaStream_t);

void launch_trunk_mask_mats(long long count, int dim, int nf, int p, int q, bool unit_diag,
                            double* mats, cudaStream_t s) {
  if (count == 0) return;
  int n = nf;
  for (int a = 0; a < dim; ++a) n *= p + 1;
  trunk_mask_mats_kernel<<<grid_for(count * n * n), 256, 0, s>>>(count, dim, nf, p, q,
                                                                 unit_diag ? 1 : 0, mats);
}

void launch_trunk_mask_vec(const LevelGeom& g, int q, double* v, cudaStream_t s) {
  trunk_mask_vec_kernel<<<grid_for(g.N), 256, 0, s>>>(g, q, v);
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
  const long long nb = (g.N + 256 * kGatherDofs - 1) / (256 * kGatherDofs);
  const int grid = (int)(nb < 65535 * 16 ? nb : 65535 * 16);
  TV tw = (TV)w;
  switch (mode) {
    case GATHER_SET: launch_pdl(gather_kernel<TV, GATHER_SET>, dim3(grid), dim3(256), 0, s, g, Y, b, out, tw); break;
    case GATHER_RESID: launch_pdl(gather_kernel<TV, GATHER_RESID>, dim3(grid), dim3(256), 0, s, g, Y, b, out, tw); break;
    case GATHER_ADD: launch_pdl(gather_kernel<TV, GATHER_ADD>, dim3(grid), dim3(256), 0, s, g, Y, b, out, tw); break;
    default: launch_pdl(gather_kernel<TV, GATHER_SCALE>, dim3(grid), dim3(256), 0, s, g, Y, b, out, tw); break;
  }
}

template <typename TV>
void launch_p_restrict(const LevelGeom& gc, const LevelGeom& gf, const TV* rf, TV* bc,
                       cudaStream_t s) {
  launch_pdl(p_transfer_kernel<TV, false>, dim3(grid_for(gc.N)), dim3(256), 0, s, gc, gf, rf, bc);
}
template <typename TV>
void launch_p_prolong_add(const LevelGeom& gc, const LevelGeom& gf, const TV* xc, TV* xf,
                          cudaStream_t s) {
  launch_pdl(p_transfer_kernel<TV, true>, dim3(grid_for(gc.N)), dim3(256), 0, s, gc, gf, xc, xf);
}
template <typename TV>
void launch_h_restrict(const LevelGeom& gc, const LevelGeom& gf, const TV* rf, TV* bc,
                       cudaStream_t s) {
  launch_pdl(h_restrict_kernel<TV>, dim3(grid_for(gc.N)), dim3(256), 0, s, gc, gf, rf, bc);
}
template <typename TV>
void launch_h_prolong_add(const LevelGeom& gc, const LevelGeom& gf, const TV* xc, TV* xf,
                          cudaStream_t s) {
  launch_pdl(h_prolong_kernel<TV>, dim3(grid_for(gf.N)), dim3(256), 0, s, gc, gf, xc, xf);
}
template <typename TV>
void launch_coarse_solve(int n, const double* L, const TV* b, TV* x, cudaStream_t s) {
  launch_pdl(coarse_solve_kernel<TV>, dim3(1), dim3(1024), 2 * n * sizeof(double), s, n, L, b, x);
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
                                   cudaStream_t, const SideStream*);                           \
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

cudaError_t read_and_clear_timeout(int* flag, cudaStream_t s) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(flag, g_stream_timeout, sizeof(int), 0,
                                            cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || *flag == 0) return e;
  const int zero = 0;
  e = cudaMemcpyToSymbolAsync(g_stream_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace fcm
