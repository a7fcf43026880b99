// Setup kernels: Gauss-Legendre rules, cell classification, cut-cell
// space-tree quadrature with penalty surfaces, and uncut-cell loads.
//
// This translation unit is compiled with -fmad=false: every geometric
// quantity that decides a classification (cell and sub-cell boxes, level-set
// values at corners, lattice points and quadrature points) is computed with
// separately rounded multiplies and adds in a fixed order, so the decisions
// are reproducible by any IEEE-754 implementation of the same formulas.
#include <algorithm>
#include <cmath>

#include "fcm_internal.h"
#include "geom.h"

namespace fcm {

namespace {

// --------------------------------------------------------------------------
// Gauss-Legendre rule (nodes ascending, weights): roots of P_n by Newton's
// method from cos(pi (i - 1/4) / (n + 1/2)), positive half mirrored.
__global__ void gauss_table_kernel(int n, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* xs = out;
  double* ws = out + n;
  int half = n / 2;
  for (int i = 1; i <= half; ++i) {
    double x = cos(M_PI * (i - 0.25) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x = x - dx;
      if (fabs(dx) <= 1e-17) break;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (x * p1 - p0) / (x * x - 1.0);
    double w = 2.0 / ((1.0 - x * x) * dp * dp);
    // i-th largest root: position n - i ascending; mirror at i - 1
    xs[n - i] = x;
    ws[n - i] = w;
    xs[i - 1] = -x;
    ws[i - 1] = w;
  }
  if (n % 2) {
    double x = 0.0;
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (x * p1 - p0) / (x * x - 1.0);
    xs[half] = 0.0;
    ws[half] = 2.0 / (dp * dp);
  }
}

__device__ void cell_box(const Problem& P, int cx, int cy, int cz, double* x0, double* x1) {
  int c[3] = {cx, cy, cz};
  for (int a = 0; a < 3; ++a) {
    if (a < P.dim) {
      double h = (P.hi[a] - P.lo[a]) / P.C[a];
      x0[a] = P.lo[a] + c[a] * h;
      x1[a] = P.lo[a] + (c[a] + 1) * h;
    } else {
      x0[a] = 0.0;
      x1[a] = 0.0;
    }
  }
}

__global__ void classify_kernel(Problem P, signed char* cls, unsigned char* faces) {
  int ncell = P.C[0] * P.C[1] * P.C[2];
  Geo G{P.geom_kind, P.dim, P.n_gparams, P.d_gparams, P.geom_complement};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    int cx = c % P.C[0], cy = (c / P.C[0]) % P.C[1], cz = c / (P.C[0] * P.C[1]);
    double x0[3], x1[3];
    cell_box(P, cx, cy, cz, x0, x1);
    cls[c] = (signed char)classify_box(G, x0, x1);
    int cc[3] = {cx, cy, cz};
    unsigned f = 0;
    for (int a = 0; a < P.dim; ++a) {
      if (cc[a] == 0) f |= 1u << (2 * a);
      if (cc[a] == P.C[a] - 1) f |= 1u << (2 * a + 1);
    }
    faces[c] = (unsigned char)f;
  }
}

// --------------------------------------------------------------------------
// 1D integrated Legendre modes: N_0 = (1-xi)/2, N_1 = (1+xi)/2,
// N_j = (P_j - P_{j-2}) / sqrt(4j-2), N_j' = sqrt((2j-1)/2) P_{j-1}.
__device__ void basis1d(int p, double xi, double* N, double* dN) {
  double Pl[kMaxP + 2];
  Pl[0] = 1.0;
  Pl[1] = xi;
  for (int k = 1; k < p; ++k) Pl[k + 1] = ((2 * k + 1) * xi * Pl[k] - k * Pl[k - 1]) / (k + 1);
  N[0] = 0.5 * (1.0 - xi);
  N[1] = 0.5 * (1.0 + xi);
  dN[0] = -0.5;
  dN[1] = 0.5;
  for (int j = 2; j <= p; ++j) {
    N[j] = (Pl[j] - Pl[j - 2]) / sqrt(4.0 * j - 2.0);
    dN[j] = sqrt((2.0 * j - 1.0) / 2.0) * Pl[j - 1];
  }
}

__device__ double source_f(const Problem& P, const double* x) {
  if (P.pde == FCM_PDE_ELASTICITY || P.source == FCM_SRC_CONST) return P.f0;
  if (P.source == FCM_SRC_SIN3) {
    double u = 1.0;
    for (int a = 0; a < P.dim; ++a) u = u * sin(M_PI * x[a]);
    return P.kappa * P.dim * (M_PI * M_PI) * u;
  }
  if (P.source == FCM_SRC_POPCORN) {
    // -kappa Lap u, u = x^3 + x y^2 + y^3 + z^4 + sin(3 (x^2 + y^2))
    const double r2 = x[0] * x[0] + x[1] * x[1];
    const double lap = 8.0 * x[0] + 6.0 * x[1] + 12.0 * x[2] * x[2] + 12.0 * cos(3.0 * r2) -
                       36.0 * r2 * sin(3.0 * r2);
    return -P.kappa * lap;
  }
  double a = P.src_a;
  return cos(a * (x[0] - 0.5)) * sin(a * (x[1] - 0.5));
}

__device__ double dirichlet_g(const Problem& P, const double* x) {
  if (P.pde == FCM_PDE_ELASTICITY || P.g == FCM_G_ZERO) return 0.0;
  if (P.g == FCM_G_SIN3) {
    double u = 1.0;
    for (int a = 0; a < P.dim; ++a) u = u * sin(M_PI * x[a]);
    return u;
  }
  if (P.g == FCM_G_POPCORN) {
    const double X = x[0], Y = x[1], Z = x[2];
    return X * X * X + X * Y * Y + Y * Y * Y + Z * Z * Z * Z + sin(3.0 * (X * X + Y * Y));
  }
  double a = P.src_a;
  return cos(a * (x[0] - 0.5)) * sin(a * (x[1] - 0.5)) / (2.0 * P.kappa * a * a);
}

// Tree node of the cut-cell space tree.
struct Node {
  double lo[3], hi[3];
  int type;  // 0 inside leaf, 1 outside leaf, 2 cut leaf (max depth), 3 interior
  int level;
};

constexpr int kThreads = 256;
constexpr int kMaxPts = 128;       // points per batch
constexpr int kMaxPairs = 40;      // accumulators per thread (n(n+1)/2 <= 10240)
constexpr int kMaxSurfPieces = 12; // 6 Kuhn tetrahedra x 2 triangles

struct PointBatch {
  double x[kMaxPts][3];
  double w[kMaxPts];        // volume: w * alpha; surface: beta * w
  double fg[kMaxPts];       // volume: f; surface: g
  double T[kMaxPts][3][2][kMaxP + 1];  // per axis: N_j, dN_j (dN scaled to physical)
};

// Evaluate the per-axis 1D tables for `np` points of the batch.
__device__ void batch_tables(PointBatch& B, int np, int dim, int p, const double* x0,
                             const double* x1) {
  for (int t = threadIdx.x; t < np * dim; t += blockDim.x) {
    int q = t / dim, a = t % dim;
    double xi = (2.0 * B.x[q][a] - (x0[a] + x1[a])) / (x1[a] - x0[a]);
    double N[kMaxP + 1], dN[kMaxP + 1];
    basis1d(p, xi, N, dN);
    double s = 2.0 / (x1[a] - x0[a]);
    for (int j = 0; j <= p; ++j) {
      B.T[q][a][0][j] = N[j];
      B.T[q][a][1][j] = dN[j] * s;
    }
  }
}

struct PairSet {
  int cnt;
  unsigned short i[kMaxPairs], j[kMaxPairs];
  double acc[kMaxPairs];
};

__device__ void mode_axes(int l, int P1, int dim, int* ja) {
  ja[0] = l % P1;
  ja[1] = dim > 1 ? (l / P1) % P1 : 0;
  ja[2] = dim > 2 ? l / (P1 * P1) : 0;
}

// K_ij += sum_q w_q grad N_i . grad N_j
__device__ void accumulate_stiffness(const PointBatch& B, int np, int dim, int P1,
                                     double kappa, PairSet& ps) {
  for (int k = 0; k < ps.cnt; ++k) {
    int ia[3], jb[3];
    mode_axes(ps.i[k], P1, dim, ia);
    mode_axes(ps.j[k], P1, dim, jb);
    double s = 0.0;
    for (int q = 0; q < np; ++q) {
      double v[3], d[3];
      for (int a = 0; a < dim; ++a) {
        v[a] = B.T[q][a][0][ia[a]] * B.T[q][a][0][jb[a]];
        d[a] = B.T[q][a][1][ia[a]] * B.T[q][a][1][jb[a]];
      }
      double gg;
      if (dim == 2)
        gg = d[0] * v[1] + v[0] * d[1];
      else
        gg = d[0] * v[1] * v[2] + v[0] * d[1] * v[2] + v[0] * v[1] * d[2];
      s += B.w[q] * gg;
    }
    ps.acc[k] += kappa * s;
  }
}

// K_IJ += sum_q w_q N_i N_j (surface / face penalty mass); for vector fields
// (I = f ns + i) only pairs of the same field couple.
__device__ void accumulate_mass(const PointBatch& B, int np, int dim, int P1, int ns,
                                PairSet& ps) {
  for (int k = 0; k < ps.cnt; ++k) {
    const int I = ps.i[k], J = ps.j[k];
    if (I / ns != J / ns) continue;
    int ia[3], jb[3];
    mode_axes(I % ns, P1, dim, ia);
    mode_axes(J % ns, P1, dim, jb);
    double s = 0.0;
    for (int q = 0; q < np; ++q) {
      double v = 1.0;
      for (int a = 0; a < dim; ++a) v *= B.T[q][a][0][ia[a]] * B.T[q][a][0][jb[a]];
      s += B.w[q] * v;
    }
    ps.acc[k] += s;
  }
}

// Isotropic linear elasticity, K_{fi,gj} += sum_q w_q (lambda N_i,f N_j,g +
// mu N_i,g N_j,f + mu delta_fg grad N_i . grad N_j): the entries of
// B^T C B for the Voigt strain operator B and isotropic C.
__device__ void accumulate_elastic(const PointBatch& B, int np, int dim, int P1, int ns,
                                   double lam, double mu, PairSet& ps) {
  for (int k = 0; k < ps.cnt; ++k) {
    const int I = ps.i[k], J = ps.j[k];
    const int f = I / ns, g = J / ns;
    int ia[3], jb[3];
    mode_axes(I % ns, P1, dim, ia);
    mode_axes(J % ns, P1, dim, jb);
    double s = 0.0;
    for (int q = 0; q < np; ++q) {
      double gi[3], gj[3];
      for (int a = 0; a < dim; ++a) {
        double vi = 1.0, vj = 1.0;
        for (int b = 0; b < dim; ++b) {
          vi *= B.T[q][b][a == b ? 1 : 0][ia[b]];
          vj *= B.T[q][b][a == b ? 1 : 0][jb[b]];
        }
        gi[a] = vi;
        gj[a] = vj;
      }
      double t = lam * gi[f] * gj[g] + mu * gi[g] * gj[f];
      if (f == g) {
        double d = 0.0;
        for (int a = 0; a < dim; ++a) d += gi[a] * gj[a];
        t += mu * d;
      }
      s += B.w[q] * t;
    }
    ps.acc[k] += s;
  }
}

// Sum factorisation of the leaf sums (FCM_QUAD_SUMFACT).  The points of a
// leaf are its tensor grid q = q0 + P q1 + P^2 q2 (P = p + 1 per axis, x
// fastest) with weights W_q = B.w[q], so every product of 1D factors in the
// pair sums contracts one axis at a time:
//   Z[v][q0 + P q1][i2, j2] = sum_q2 W_q A2(si, q2, i2) A2(sj, q2, j2),
//   Y[u][q0][(i1, i2), (j1, j2)] = sum_q1 Z[..][q0 + P q1][i2, j2] A1(.., q1, i1) A1(.., q1, j1),
//   K_IJ += sum_q0 Y[..][q0][(i1, i2), (j1, j2)] A0(.., q0, i0) A0(.., q0, j0),
// with A_a(s, q, m) the mode m (s = 1: its derivative) at the axis-a
// coordinate of the leaf's q-th Gauss point (read from B.T).  A 2D problem
// has one point and one mode (value 1, derivative 0) on axis 2.  Poisson
// needs Y for no derivative on axes 1 and 2 and for one derivative on either;
// elasticity one Y per (f, g) for the integrals of d_f N_i d_g N_j.  Every
// thread of the block calls this (it synchronises).
__host__ __device__ inline int sf_doubles(int dim, int P, bool elastic) {
  const int P2 = dim == 3 ? P : 1, M12 = P * P2;
  return 6 * P * P + 4 * P * P * P2 * P2 + (elastic ? dim * dim : 2) * P * M12 * M12;
}

__device__ void sf_accumulate(const PointBatch& B, double* sfx, int dim, int P, int ns,
                              bool elastic, double lam, double mu, double kappa, PairSet& ps) {
  const int P2 = dim == 3 ? P : 1;  // points and modes on axis 2
  const int M12 = P * P2;           // modes on axes 1 and 2: r = i1 + P i2
  const int PP = P * P, Z2 = P2 * P2;
  double* A = sfx;                  // [axis][s][q][m]: 3 x 2 x P x P
  double* Z = A + 6 * PP;           // [v = si + 2 sj][q0 + P q1][i2 + P2 j2]
  double* Y = Z + 4 * PP * Z2;      // [u][q0][r][c]
  const int ny = P * M12 * M12;
  for (int t = threadIdx.x; t < 6 * PP; t += blockDim.x) {
    const int m = t % P, q = (t / P) % P, sd = (t / PP) % 2, a = t / (2 * PP);
    double v;
    if (a < dim)
      v = B.T[a == 0 ? q : (a == 1 ? q * P : q * PP)][a][sd][m];
    else
      v = (sd == 0 && q == 0 && m == 0) ? 1.0 : 0.0;
    A[t] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 4 * PP * Z2; t += blockDim.x) {
    const int e = t % Z2, q01 = (t / Z2) % PP, v = t / (Z2 * PP);
    const int i2 = e % P2, j2 = e / P2;
    const double* ai = A + (4 + (v & 1)) * PP;
    const double* aj = A + (4 + (v >> 1)) * PP;
    double z = 0.0;
    for (int q2 = 0; q2 < P2; ++q2) z += B.w[q01 + PP * q2] * ai[q2 * P + i2] * aj[q2 * P + j2];
    Z[t] = z;
  }
  __syncthreads();
  const int nu = elastic ? dim * dim : 2;
  for (int t = threadIdx.x; t < nu * ny; t += blockDim.x) {
    const int w = t % ny, u = t / ny;
    const int c = w % M12, r = (w / M12) % M12, q0 = w / (M12 * M12);
    const int i1 = r % P, i2 = r / P, j1 = c % P, j2 = c / P;
    const int e = i2 + P2 * j2;
    double y = 0.0;
    if (!elastic) {
      // u = 0: no derivative on axes 1, 2; u = 1: one derivative on axis 1 or 2
      const double* a10 = A + 2 * PP;
      const double* a11 = A + 3 * PP;
      for (int q1 = 0; q1 < P; ++q1) {
        const double z0 = Z[(q0 + P * q1) * Z2 + e];
        const double v0 = a10[q1 * P + i1] * a10[q1 * P + j1];
        if (u == 0) {
          y += z0 * v0;
        } else {
          const double z1 = Z[(3 * PP + q0 + P * q1) * Z2 + e];
          y += z0 * (a11[q1 * P + i1] * a11[q1 * P + j1]) + z1 * v0;
        }
      }
    } else {
      const int f = u / dim, g = u % dim;
      const int v = (f == 2 ? 1 : 0) + 2 * (g == 2 ? 1 : 0);
      const double* ai = A + (2 + (f == 1 ? 1 : 0)) * PP;
      const double* aj = A + (2 + (g == 1 ? 1 : 0)) * PP;
      for (int q1 = 0; q1 < P; ++q1)
        y += Z[(v * PP + q0 + P * q1) * Z2 + e] * ai[q1 * P + i1] * aj[q1 * P + j1];
    }
    Y[t] = y;
  }
  __syncthreads();
  for (int k = 0; k < ps.cnt; ++k) {
    const int I = ps.i[k], J = ps.j[k];
    double s = 0.0;
    if (!elastic) {
      const int i0 = I % P, r = I / P, j0 = J % P, c = J / P;
      for (int q0 = 0; q0 < P; ++q0) {
        const int o = (q0 * M12 + r) * M12 + c;
        s += Y[o] * (A[PP + q0 * P + i0] * A[PP + q0 * P + j0]) +
             Y[ny + o] * (A[q0 * P + i0] * A[q0 * P + j0]);
      }
      ps.acc[k] += kappa * s;
    } else {
      const int f = I / ns, g = J / ns, i = I % ns, j = J % ns;
      const int i0 = i % P, r = i / P, j0 = j % P, c = j / P;
      const int sf0 = f == 0 ? 1 : 0, sg0 = g == 0 ? 1 : 0;
      for (int q0 = 0; q0 < P; ++q0) {
        const int o = (q0 * M12 + r) * M12 + c;
        double t = lam * Y[(f * dim + g) * ny + o] * (A[sf0 * PP + q0 * P + i0] * A[sg0 * PP + q0 * P + j0]) +
                   mu * Y[(g * dim + f) * ny + o] * (A[sg0 * PP + q0 * P + i0] * A[sf0 * PP + q0 * P + j0]);
        if (f == g)
          for (int a = 0; a < dim; ++a) {
            const int sa = a == 0 ? 1 : 0;
            t += mu * Y[(a * dim + a) * ny + o] * (A[sa * PP + q0 * P + i0] * A[sa * PP + q0 * P + j0]);
          }
        s += t;
      }
      ps.acc[k] += s;
    }
  }
}

// b_i += sum_q w_q fg_q N_i
__device__ void accumulate_load(const PointBatch& B, int np, int dim, int P1, int n,
                                double* bacc) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int ia[3];
    mode_axes(i, P1, dim, ia);
    double s = 0.0;
    for (int q = 0; q < np; ++q) {
      double v = 1.0;
      for (int a = 0; a < dim; ++a) v *= B.T[q][a][0][ia[a]];
      s += B.w[q] * B.fg[q] * v;
    }
    bacc[i] += s;
  }
}

__device__ void edge_point(const double (*v)[3], const double* psi, int i, int j, int dim,
                           double* out) {
  double t = psi[i] / (psi[i] - psi[j]);
  for (int a = 0; a < dim; ++a) out[a] = v[i][a] + t * (v[j][a] - v[i][a]);
}

// Marching simplices on a leaf box (thread 0).  Returns the piece count;
// each piece is 2 (2D) or 3 (3D) points.
__device__ int marching(const Geo& G, int dim, const double* lo, const double* hi,
                        double (*pc)[3][3]) {
  double v[8][3];
  double psi[8];
  int nc = 1 << dim;
  for (int k = 0; k < nc; ++k) {
    for (int a = 0; a < 3; ++a) v[k][a] = a < dim ? (((k >> a) & 1) ? hi[a] : lo[a]) : 0.0;
    psi[k] = levelset(G, v[k]);
  }
  const int perm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int perm2[2][2] = {{0, 1}, {1, 0}};
  int npc = 0;
  int nperm = dim == 3 ? 6 : 2;
  for (int pi = 0; pi < nperm; ++pi) {
    int seq[4];
    int k = 0;
    seq[0] = 0;
    for (int s = 0; s < dim; ++s) {
      int a = dim == 3 ? perm3[pi][s] : perm2[pi][s];
      k |= 1 << a;
      seq[s + 1] = k;
    }
    int ins[4], outs[4], ni = 0, no = 0;
    for (int s = 0; s <= dim; ++s) {
      if (psi[seq[s]] <= 0.0)
        ins[ni++] = seq[s];
      else
        outs[no++] = seq[s];
    }
    if (ni == 0 || no == 0) continue;
    if (dim == 2) {
      if (ni == 1) {
        edge_point(v, psi, ins[0], outs[0], 2, pc[npc][0]);
        edge_point(v, psi, ins[0], outs[1], 2, pc[npc][1]);
      } else {
        edge_point(v, psi, ins[0], outs[0], 2, pc[npc][0]);
        edge_point(v, psi, ins[1], outs[0], 2, pc[npc][1]);
      }
      ++npc;
    } else {
      if (ni == 1) {
        for (int s = 0; s < 3; ++s) edge_point(v, psi, ins[0], outs[s], 3, pc[npc][s]);
        ++npc;
      } else if (ni == 3) {
        for (int s = 0; s < 3; ++s) edge_point(v, psi, ins[s], outs[0], 3, pc[npc][s]);
        ++npc;
      } else {
        double q0[3], q1[3], q2[3], q3[3];
        edge_point(v, psi, ins[0], outs[0], 3, q0);
        edge_point(v, psi, ins[0], outs[1], 3, q1);
        edge_point(v, psi, ins[1], outs[1], 3, q2);
        edge_point(v, psi, ins[1], outs[0], 3, q3);
        for (int a = 0; a < 3; ++a) {
          pc[npc][0][a] = q0[a];
          pc[npc][1][a] = q1[a];
          pc[npc][2][a] = q2[a];
          pc[npc + 1][0][a] = q0[a];
          pc[npc + 1][1][a] = q2[a];
          pc[npc + 1][2][a] = q3[a];
        }
        npc += 2;
      }
    }
  }
  return npc;
}

struct ElemShared {
  PointBatch B;
  double pieces[kMaxSurfPieces][3][3];
  int npieces;
  int nnodes;
  int seg_begin, seg_end;
  int scan[kThreads];
  double x0[3], x1[3];
  double gauss[2 * (kMaxP + 1)];
};

// Start of the sum-factorisation scratch behind ElemShared (16-byte aligned).
__host__ __device__ constexpr size_t sf_offset() { return (sizeof(ElemShared) + 15) / 16 * 16; }

// One CTA per own cell: volume terms on the space-tree leaves, penalty on
// the marching-simplex surface of cut leaves, box-face penalty and traction.
// Poisson (n = (p+1)^d) or isotropic elasticity (n = d (p+1)^d, fields
// stacked).
__global__ void __launch_bounds__(kThreads) element_own_kernel(
    Problem P, const double* gauss, int ncell, const int* cells, double* Kout, double* bout,
    Node* scratch, int max_nodes, int sf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ElemShared& S = *reinterpret_cast<ElemShared*>(smem_raw);
  double* sfx = reinterpret_cast<double*>(smem_raw + sf_offset());  // sum factorisation
  const int dim = P.dim, p = P.p, P1 = p + 1;
  int ns = 1;
  for (int a = 0; a < dim; ++a) ns *= P1;
  const int n = P.nf * ns;
  const int npairs = n * (n + 1) / 2;
  const bool elastic = P.pde == FCM_PDE_ELASTICITY;
  const double lam = P.E * P.nu / ((1.0 + P.nu) * (1.0 - 2.0 * P.nu));
  const double mu = P.E / (2.0 * (1.0 + P.nu));
  Geo G{P.geom_kind, dim, P.n_gparams, P.d_gparams, P.geom_complement};
  const int nq1 = P1;  // points per axis
  int Qleaf = 1;
  for (int a = 0; a < dim; ++a) Qleaf *= nq1;

  for (int t = threadIdx.x; t < 2 * P1; t += blockDim.x) S.gauss[t] = gauss[t];

  for (int ci = blockIdx.x; ci < ncell; ci += gridDim.x) {
    const int cell = cells[ci];
    const bool ref = cell < 0;
    int cx = 0, cy = 0, cz = 0;
    if (!ref) {
      cx = cell % P.C[0];
      cy = (cell / P.C[0]) % P.C[1];
      cz = cell / (P.C[0] * P.C[1]);
    }
    Node* nodes = scratch + (size_t)blockIdx.x * max_nodes;
    if (threadIdx.x == 0) {
      cell_box(P, cx, cy, cz, S.x0, S.x1);
      Node r;
      for (int a = 0; a < 3; ++a) {
        r.lo[a] = S.x0[a];
        r.hi[a] = S.x1[a];
      }
      r.level = 0;
      r.type = ref ? 0 : -1;
      nodes[0] = r;
      S.nnodes = 1;
      S.seg_begin = 0;
      S.seg_end = 1;
    }
    __syncthreads();
    // breadth-first space tree with deterministic child order
    while (S.seg_begin < S.seg_end) {
      int b0 = S.seg_begin, b1 = S.seg_end;
      for (int base = b0; base < b1; base += blockDim.x) {
        int idx = base + threadIdx.x;
        int split = 0;
        if (idx < b1) {
          Node& nd = nodes[idx];
          if (nd.type < 0) {
            int c = classify_box(G, nd.lo, nd.hi);
            if (c != CLS_CUT)
              nd.type = c;  // 0 inside / 1 outside
            else if (nd.level == P.quad_depth)
              nd.type = 2;
            else {
              nd.type = 3;
              split = 1;
            }
          }
        }
        S.scan[threadIdx.x] = split;
        __syncthreads();
        // inclusive scan (Hillis-Steele) of split flags
        for (int off = 1; off < blockDim.x; off <<= 1) {
          int v = threadIdx.x >= off ? S.scan[threadIdx.x - off] : 0;
          __syncthreads();
          S.scan[threadIdx.x] += v;
          __syncthreads();
        }
        int nch = 1 << dim;
        int before = S.scan[threadIdx.x] - split;
        int total = S.scan[blockDim.x - 1];
        if (split) {
          Node nd = nodes[idx];
          double mid[3];
          for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (nd.lo[a] + nd.hi[a]);
          for (int k = 0; k < nch; ++k) {
            Node ch;
            for (int a = 0; a < 3; ++a) {
              bool up = a < dim && ((k >> a) & 1);
              ch.lo[a] = up ? mid[a] : nd.lo[a];
              ch.hi[a] = (a < dim && !up) ? mid[a] : nd.hi[a];
            }
            ch.level = nd.level + 1;
            ch.type = -1;
            int slot = S.nnodes + before * nch + k;
            if (slot < max_nodes) nodes[slot] = ch;
          }
        }
        __syncthreads();
        if (threadIdx.x == 0) S.nnodes = min(S.nnodes + total * nch, max_nodes);
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        S.seg_begin = b1;
        S.seg_end = S.nnodes;
      }
      __syncthreads();
    }

    // pair accumulators
    PairSet ps;
    ps.cnt = 0;
    for (int k = threadIdx.x; k < npairs && ps.cnt < kMaxPairs; k += blockDim.x) {
      int i = 0, rem = k;
      while (rem >= n - i) {
        rem -= n - i;
        ++i;
      }
      ps.i[ps.cnt] = (unsigned short)i;
      ps.j[ps.cnt] = (unsigned short)(i + rem);
      ps.acc[ps.cnt] = 0.0;
      ++ps.cnt;
    }
    double bacc[4] = {0.0, 0.0, 0.0, 0.0};  // modes threadIdx.x + k * blockDim.x
    // volume leaves
    const int nn = S.nnodes;
    for (int li = 0; li < nn; ++li) {
      Node nd = nodes[li];
      if (nd.type == 3) continue;
      double mids[3], hds[3];
      for (int a = 0; a < dim; ++a) {
        mids[a] = 0.5 * (nd.lo[a] + nd.hi[a]);
        hds[a] = 0.5 * (nd.hi[a] - nd.lo[a]);
      }
      for (int q0 = 0; q0 < Qleaf; q0 += kMaxPts) {
        int np = min(kMaxPts, Qleaf - q0);
        for (int t = threadIdx.x; t < np; t += blockDim.x) {
          int q = q0 + t;
          int ia[3];
          mode_axes(q, nq1, dim, ia);
          double w = 1.0;
          for (int a = 0; a < dim; ++a) {
            S.B.x[t][a] = mids[a] + hds[a] * S.gauss[ia[a]];
            double wa = hds[a] * S.gauss[P1 + ia[a]];
            w = a == 0 ? wa : w * wa;
          }
          double alpha;
          if (nd.type == 0)
            alpha = 1.0;
          else if (nd.type == 1)
            alpha = P.alpha;
          else
            alpha = levelset(G, S.B.x[t]) <= 0.0 ? 1.0 : P.alpha;
          S.B.w[t] = w * alpha;
          S.B.fg[t] = source_f(P, S.B.x[t]);
        }
        __syncthreads();
        batch_tables(S.B, np, dim, p, S.x0, S.x1);
        __syncthreads();
        if (sf)  // the leaf's points are one batch (np == Qleaf)
          sf_accumulate(S.B, sfx, dim, P1, ns, elastic, lam, mu, P.kappa, ps);
        else if (elastic)
          accumulate_elastic(S.B, np, dim, P1, ns, lam, mu, ps);
        else
          accumulate_stiffness(S.B, np, dim, P1, P.kappa, ps);
        double bl[4] = {0, 0, 0, 0};
        {
          // load with the same tables (every field gets the same body load)
          for (int k = 0; k < 4; ++k) {
            int i = threadIdx.x + k * blockDim.x;
            if (i >= n) break;
            int ia[3];
            mode_axes(i % ns, P1, dim, ia);
            double s = 0.0;
            for (int q = 0; q < np; ++q) {
              double v = 1.0;
              for (int a = 0; a < dim; ++a) v *= S.B.T[q][a][0][ia[a]];
              s += S.B.w[q] * S.B.fg[q] * v;
            }
            bl[k] = s;
          }
        }
        for (int k = 0; k < 4; ++k) bacc[k] += bl[k];
        __syncthreads();
      }
      // immersed penalty surface on cut leaves
      if (nd.type == 2 && P.dirichlet == FCM_DIR_LEVELSET && !ref) {
        if (threadIdx.x == 0) S.npieces = marching(G, dim, nd.lo, nd.hi, S.pieces);
        __syncthreads();
        const int npc = S.npieces;
        const int ppp = dim == 2 ? P1 : P1 * P1;  // points per piece
        for (int pcs = 0; pcs < npc; ++pcs) {
          for (int t = threadIdx.x; t < ppp; t += blockDim.x) {
            double u[2], wu[2];
            int ii = dim == 2 ? t : t / P1, jj = dim == 2 ? 0 : t % P1;
            u[0] = 0.5 * (S.gauss[ii] + 1.0);
            wu[0] = 0.5 * S.gauss[P1 + ii];
            u[1] = 0.5 * (S.gauss[jj] + 1.0);
            wu[1] = 0.5 * S.gauss[P1 + jj];
            const double* A = S.pieces[pcs][0];
            const double* Bp = S.pieces[pcs][1];
            double w;
            if (dim == 2) {
              double dx = Bp[0] - A[0], dy = Bp[1] - A[1];
              double L = sqrt(dx * dx + dy * dy);
              S.B.x[t][0] = A[0] + u[0] * dx;
              S.B.x[t][1] = A[1] + u[0] * dy;
              w = wu[0] * L;
            } else {
              const double* Cp = S.pieces[pcs][2];
              double e1[3], e2[3];
              for (int a = 0; a < 3; ++a) {
                e1[a] = Bp[a] - A[a];
                e2[a] = Cp[a] - Bp[a];
              }
              double c0 = e1[1] * e2[2] - e1[2] * e2[1];
              double c1 = e1[2] * e2[0] - e1[0] * e2[2];
              double c2 = e1[0] * e2[1] - e1[1] * e2[0];
              double J = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
              for (int a = 0; a < 3; ++a) S.B.x[t][a] = A[a] + u[0] * e1[a] + (u[0] * u[1]) * e2[a];
              w = wu[0] * wu[1] * u[0] * J;
            }
            S.B.w[t] = P.beta * w;
            S.B.fg[t] = dirichlet_g(P, S.B.x[t]);
          }
          __syncthreads();
          batch_tables(S.B, ppp, dim, p, S.x0, S.x1);
          __syncthreads();
          accumulate_mass(S.B, ppp, dim, P1, ns, ps);
          for (int k = 0; k < 4; ++k) {
            int i = threadIdx.x + k * blockDim.x;
            if (i >= n) break;
            int ia[3];
            mode_axes(i % ns, P1, dim, ia);
            double s = 0.0;
            for (int q = 0; q < ppp; ++q) {
              double v = 1.0;
              for (int a = 0; a < dim; ++a) v *= S.B.T[q][a][0][ia[a]];
              s += S.B.w[q] * S.B.fg[q] * v;
            }
            bacc[k] += s;
          }
          __syncthreads();
        }
      }
    }
    // box faces: Dirichlet penalty (K and b) and traction (b only)
    if (!ref) {
      int cc[3] = {cx, cy, cz};
      for (int face = 0; face < 2 * dim; ++face) {
        int a = face / 2, sd = face % 2;
        bool on = sd == 0 ? cc[a] == 0 : cc[a] == P.C[a] - 1;
        const bool dir = P.dirichlet == FCM_DIR_FACES && ((P.dir_faces >> face) & 1u);
        const bool tra = P.traction_face == face;
        if (!on || (!dir && !tra)) continue;
        int nfp = 1;
        for (int b = 0; b < dim - 1; ++b) nfp *= P1;
        for (int t = threadIdx.x; t < nfp; t += blockDim.x) {
          double w = 1.0;
          int rem = t;
          for (int b = 0; b < dim; ++b) {
            if (b == a) {
              S.B.x[t][b] = sd ? S.x1[b] : S.x0[b];
              continue;
            }
            int ib = rem % P1;
            rem /= P1;
            double mid = 0.5 * (S.x0[b] + S.x1[b]);
            double hd = 0.5 * (S.x1[b] - S.x0[b]);
            S.B.x[t][b] = mid + hd * S.gauss[ib];
            w = w * (hd * S.gauss[P1 + ib]);
          }
          S.B.w[t] = w;
          S.B.fg[t] = dirichlet_g(P, S.B.x[t]);
        }
        __syncthreads();
        batch_tables(S.B, nfp, dim, p, S.x0, S.x1);
        __syncthreads();
        if (dir) {
          for (int t = threadIdx.x; t < nfp; t += blockDim.x) S.B.w[t] *= P.beta;
          __syncthreads();
          accumulate_mass(S.B, nfp, dim, P1, ns, ps);
        }
        for (int k = 0; k < 4; ++k) {
          int i = threadIdx.x + k * blockDim.x;
          if (i >= n) break;
          int ia[3];
          mode_axes(i % ns, P1, dim, ia);
          const int fld = i / ns;
          double sdir = 0.0, stra = 0.0;
          for (int q = 0; q < nfp; ++q) {
            double v = 1.0;
            for (int b = 0; b < dim; ++b) v *= S.B.T[q][b][0][ia[b]];
            sdir += S.B.w[q] * S.B.fg[q] * v;
            stra += S.B.w[q] * v;
          }
          if (dir) bacc[k] += sdir;
          // traction: int t_f N_i over the face (w not scaled by beta then)
          if (tra && !dir) bacc[k] += P.traction[fld] * stra;
        }
        __syncthreads();
      }
    }
    // write K (symmetric) and b
    double* K = Kout + (size_t)ci * n * n;
    for (int k = 0; k < ps.cnt; ++k) {
      double v = ps.acc[k];
      K[(size_t)ps.i[k] * n + ps.j[k]] = v;
      K[(size_t)ps.j[k] * n + ps.i[k]] = v;
    }
    for (int k = 0; k < 4; ++k) {
      int i = threadIdx.x + k * blockDim.x;
      if (i < n) bout[(size_t)ci * n + i] = bacc[k];
    }
    __syncthreads();
  }
}

// Uncut cells: b_c = alpha_c int f N with the (p+1)^d Gauss rule.  One warp
// per cell.
__global__ void load_uncut_kernel(Problem P, const double* gauss, int ncell, const int* cells,
                                  const signed char* cls, double* Bcells) {
  const int dim = P.dim, p = P.p, P1 = p + 1;
  int ns = 1;
  for (int a = 0; a < dim; ++a) ns *= P1;
  const int n = P.nf * ns;
  int Q = ns;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int ci = warp; ci < ncell; ci += nwarps) {
    int cell = cells[ci];
    int cx = cell % P.C[0], cy = (cell / P.C[0]) % P.C[1], cz = cell / (P.C[0] * P.C[1]);
    double x0[3], x1[3];
    cell_box(P, cx, cy, cz, x0, x1);
    double alpha = cls[cell] == CLS_INSIDE ? 1.0 : P.alpha;
    double mids[3], hds[3];
    for (int a = 0; a < dim; ++a) {
      mids[a] = 0.5 * (x0[a] + x1[a]);
      hds[a] = 0.5 * (x1[a] - x0[a]);
    }
    for (int i = lane; i < n; i += 32) {
      int ia[3];
      mode_axes(i % ns, P1, dim, ia);
      double s = 0.0;
      for (int q = 0; q < Q; ++q) {
        int qa[3];
        mode_axes(q, P1, dim, qa);
        double x[3] = {0, 0, 0};
        double w = 1.0, v = 1.0;
        for (int a = 0; a < dim; ++a) {
          x[a] = mids[a] + hds[a] * gauss[qa[a]];
          double wa = hds[a] * gauss[P1 + qa[a]];
          w = a == 0 ? wa : w * wa;
          double N[kMaxP + 1], dN[kMaxP + 1];
          double xi = (2.0 * x[a] - (x0[a] + x1[a])) / (x1[a] - x0[a]);
          basis1d(p, xi, N, dN);
          v *= N[ia[a]];
        }
        s += (w * alpha) * source_f(P, x) * v;
      }
      Bcells[(size_t)i * (P.C[0] * P.C[1] * P.C[2]) + cell] = s;  // [local][cell]
    }
  }
}

// Rows src[r][l] of own cells into the [local][cell] per-cell array.
__global__ void scatter_rows_kernel(int nrows, const int* cells, const double* src, int nloc,
                                    long long ncells, double* dst) {
  long long tot = (long long)nrows * nloc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / nloc), l = (int)(t % nloc);
    dst[(size_t)l * ncells + cells[r]] = src[t];
  }
}

}  // namespace

void launch_gauss_table(int n, double* out, cudaStream_t s) {
  gauss_table_kernel<<<1, 1, 0, s>>>(n, out);
}

void launch_classify(const Problem& P, signed char* cls, unsigned char* faces, cudaStream_t s) {
  int ncell = P.C[0] * P.C[1] * P.C[2];
  int blocks = (ncell + 255) / 256;
  classify_kernel<<<blocks, 256, 0, s>>>(P, cls, faces);
}

void launch_element_own(const Problem& P, const double* gauss, int ncell, const int* cells,
                        double* K, double* bvec, int* leaf_scratch, int max_nodes,
                        cudaStream_t s) {
  if (ncell == 0) return;
  int grid = ncell < 2048 ? ncell : 2048;
  // sum factorisation when a leaf's (p+1)^d points are one batch
  int ns = 1;
  for (int a = 0; a < P.dim; ++a) ns *= P.p + 1;
  const bool elastic = P.pde == FCM_PDE_ELASTICITY;
  const int sf = P.sumfact && ns <= kMaxPts ? 1 : 0;
  size_t smem = sf ? sf_offset() + sizeof(double) * sf_doubles(P.dim, P.p + 1, elastic)
                   : sizeof(ElemShared);
  static const bool attr = [] {
    // the largest scratch of the supported cases: (p+1)^d <= kMaxPts points
    // and at most 128 DOFs per cell
    int most = 0;
    for (int dim = 2; dim <= 3; ++dim)
      for (int P1 = 2; P1 <= kMaxP + 1; ++P1) {
        int q = 1;
        for (int a = 0; a < dim; ++a) q *= P1;
        if (q > kMaxPts) continue;
        most = std::max(most, sf_doubles(dim, P1, false));
        if (dim * q <= 128) most = std::max(most, sf_doubles(dim, P1, true));
      }
    cudaFuncSetAttribute(element_own_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sf_offset() + sizeof(double) * most));
    return true;
  }();
  (void)attr;
  element_own_kernel<<<grid, kThreads, smem, s>>>(P, gauss, ncell, cells, K, bvec,
                                                  reinterpret_cast<Node*>(leaf_scratch),
                                                  max_nodes, sf);
}

size_t element_scratch_bytes(int ncell, int max_nodes) {
  int grid = ncell < 2048 ? ncell : 2048;
  return (size_t)grid * max_nodes * sizeof(Node);
}

void launch_load_uncut(const Problem& P, const double* gauss, int ncell, const int* cells,
                       const signed char* cls, double* Bcells, cudaStream_t s) {
  if (ncell == 0) return;
  int blocks = (ncell + 7) / 8;
  if (blocks > 4096) blocks = 4096;
  load_uncut_kernel<<<blocks, 256, 0, s>>>(P, gauss, ncell, cells, cls, Bcells);
}

void launch_scatter_rows(int n, const int* cells, const double* src, int nloc, long long ncells,
                         double* Bcells, cudaStream_t s) {
  if (n == 0) return;
  long long tot = (long long)n * nloc;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  scatter_rows_kernel<<<blocks, 256, 0, s>>>(n, cells, src, nloc, ncells, Bcells);
}

}  // namespace fcm
