// Level-set geometry and box classification (Sec. 2.1: Omega_phys =
// {psi <= 0}), shared by the device setup (setup_geom.cu) and the host-side
// overlay builder (mlhp.cu).  Both translation units evaluate these formulas
// with separately rounded multiplies and adds in the order written
// (-fmad=false on the device, -ffp-contract=off on the host), so every
// classification matches a plain IEEE-754 evaluation of the same formulas.
#pragma once

#include <cmath>

#include "fcm_internal.h"

#ifdef __CUDACC__
#define FCM_HD __host__ __device__
#else
#define FCM_HD
#endif

namespace fcm {

struct Geo {
  int kind, dim, n;
  const double* prm;
  int complement;  // 1: the physical side is {psi >= 0}
};

FCM_HD inline double levelset_kind(const Geo& G, const double* x);
FCM_HD inline int classify_box_kind(const Geo& G, const double* lo, const double* hi);

// psi of the physical domain: the kind's psi, negated (exactly) for a
// complement domain.
FCM_HD inline double levelset(const Geo& G, const double* x) {
  const double v = levelset_kind(G, x);
  return G.complement ? -v : v;
}

// Box class of the physical domain: a complement domain swaps inside and
// outside (cut boxes stay cut).
FCM_HD inline int classify_box(const Geo& G, const double* lo, const double* hi) {
  const int c = classify_box_kind(G, lo, hi);
  if (!G.complement) return c;
  return c == CLS_INSIDE ? CLS_OUTSIDE : (c == CLS_OUTSIDE ? CLS_INSIDE : c);
}

FCM_HD inline double levelset_kind(const Geo& G, const double* x) {
  if (G.kind == FCM_GEOM_NONE) return -1.0;
  if (G.kind == FCM_GEOM_BALL) {
    const double* c = G.prm;
    double r = G.prm[G.dim];
    double s = (x[0] - c[0]) * (x[0] - c[0]);
    for (int a = 1; a < G.dim; ++a) s = s + (x[a] - c[a]) * (x[a] - c[a]);
    return sqrt(s) - r;
  }
  if (G.kind == FCM_GEOM_VOIDS) {
    double out = -INFINITY;
    int nb = G.n / 4;
    for (int k = 0; k < nb; ++k) {
      const double* c = G.prm + 4 * k;
      double s = (x[0] - c[0]) * (x[0] - c[0]);
      for (int a = 1; a < G.dim; ++a) s = s + (x[a] - c[a]) * (x[a] - c[a]);
      double v = c[3] - sqrt(s);
      out = k == 0 ? v : fmax(out, v);
    }
    return out;
  }
  if (G.kind == FCM_GEOM_POPCORN) {
    // r0 A sigma, then the bump centres
    const double r0 = G.prm[0], amp = G.prm[1], sig2 = G.prm[2] * G.prm[2];
    double s = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double out = sqrt(s) - r0;
    const int nc = (G.n - 3) / 3;
    for (int k = 0; k < nc; ++k) {
      const double* c = G.prm + 3 + 3 * k;
      double d2 = (x[0] - c[0]) * (x[0] - c[0]) + (x[1] - c[1]) * (x[1] - c[1]) +
                  (x[2] - c[2]) * (x[2] - c[2]);
      out = out - amp * exp(-d2 / sig2);
    }
    return out;
  }
  // ellipsoid: c(3) a(3) R(3x3 row-major)
  const double* c = G.prm;
  const double* ax = G.prm + 3;
  const double* R = G.prm + 6;
  double dx0 = x[0] - c[0], dx1 = x[1] - c[1], dx2 = x[2] - c[2];
  double q = 0.0;
  for (int i = 0; i < 3; ++i) {
    double y = R[0 * 3 + i] * dx0 + R[1 * 3 + i] * dx1 + R[2 * 3 + i] * dx2;
    double t = y / ax[i];
    q = i == 0 ? t * t : q + t * t;
  }
  return sqrt(q) - 1.0;
}

FCM_HD inline void ball_dist2(int dim, const double* lo, const double* hi, const double* c,
                           double& dmin2, double& dmax2) {
  dmin2 = 0.0;
  dmax2 = 0.0;
  for (int a = 0; a < dim; ++a) {
    double l = lo[a] - c[a];
    double u = hi[a] - c[a];
    double nr = 0.0;
    if (l > 0.0)
      nr = l;
    else if (u < 0.0)
      nr = -u;
    double fr = fmax(fabs(l), fabs(u));
    dmin2 = dmin2 + nr * nr;
    dmax2 = dmax2 + fr * fr;
  }
}

FCM_HD inline int classify_box_kind(const Geo& G, const double* lo, const double* hi) {
  if (G.kind == FCM_GEOM_NONE) return CLS_INSIDE;
  if (G.kind == FCM_GEOM_BALL) {
    double r = G.prm[G.dim];
    double dmin2, dmax2;
    ball_dist2(G.dim, lo, hi, G.prm, dmin2, dmax2);
    double r2 = r * r;
    if (dmax2 <= r2) return CLS_INSIDE;
    if (dmin2 >= r2) return CLS_OUTSIDE;
    return CLS_CUT;
  }
  if (G.kind == FCM_GEOM_VOIDS) {
    bool clear = true;
    int nb = G.n / 4;
    for (int k = 0; k < nb; ++k) {
      double dmin2, dmax2;
      ball_dist2(G.dim, lo, hi, G.prm + 4 * k, dmin2, dmax2);
      double r = G.prm[4 * k + 3];
      double r2 = r * r;
      if (dmax2 <= r2) return CLS_OUTSIDE;
      if (dmin2 < r2) clear = false;
    }
    return clear ? CLS_INSIDE : CLS_CUT;
  }
  bool any_in = false, any_out = false;
  for (int kz = 0; kz < 5; ++kz)
    for (int ky = 0; ky < 5; ++ky)
      for (int kx = 0; kx < 5; ++kx) {
        int k[3] = {kx, ky, kz};
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = lo[a] + (k[a] * 0.25) * (hi[a] - lo[a]);
        double v = levelset_kind(G, x);
        if (v <= 0.0)
          any_in = true;
        else
          any_out = true;
      }
  if (!any_out) return CLS_INSIDE;
  if (!any_in) return CLS_OUTSIDE;
  return CLS_CUT;
}

}  // namespace fcm
