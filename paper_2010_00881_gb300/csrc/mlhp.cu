// Multi-level hp overlay topology (Sec. 2.2), built on the host.
//
// Level 0 is the base grid; an element of level k < K cut by the geometry is
// overlaid by its 2^d bisection children (level k+1).  Every element carries
// the (p+1)^d tensor modes on its own box; a mode belongs to the topological
// component of its level's lattice with doubled coordinates t_a = 2 e_a
// (left node), 2 e_a + 2 (right node) or 2 e_a + 1 (bubble).  Activation:
//   R1  a component of level k >= 1 on the boundary of the refined zone (some
//       in-box lattice cell of level k around it is not an element; box
//       faces do not count) is inactive;
//   R2  a vertex of level k >= 1 with every lattice node index even (the
//       position of a level k-1 vertex) is inactive;
//   R3  edge, face and interior functions of level k are active only if the
//       component belongs to a leaf element.
// The active functions are numbered by level, then component (x fastest, z
// slowest), then bubble degrees (first odd axis fastest).  Each leaf lists
// the functions supported on it (its ancestors' active modes, ancestors from
// the base down, local modes x fastest: the row order of its element
// matrix).  Each base node lists the functions touching the base cells
// around it (the patchwise additive Schwarz block of Sec. 3.3.1).
//
// Host code only; compiled with -ffp-contract=off so that the refinement
// decisions (box classification of geom.h) round like a plain IEEE-754
// evaluation.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "fcm_internal.h"
#include "geom.h"

namespace {

constexpr int kBits = 21;                       // bits per packed coordinate
constexpr long long kMaxLattice = 1LL << 19;    // doubled coordinates < 2^20
constexpr int kMaxOverlay = 10;

inline uint64_t pack(const int* v) {
  return (uint64_t)v[0] | ((uint64_t)v[1] << kBits) | ((uint64_t)v[2] << (2 * kBits));
}
inline void unpack(uint64_t k, int* v) {
  const uint64_t m = (1ULL << kBits) - 1;
  v[0] = (int)(k & m);
  v[1] = (int)((k >> kBits) & m);
  v[2] = (int)((k >> (2 * kBits)) & m);
}
inline int mode_position(int e, int j) { return j == 0 ? 2 * e : (j == 1 ? 2 * e + 2 : 2 * e + 1); }

struct Invalid {
  std::string msg;
};

}  // namespace

struct fcm_mlhp {
  int dim = 0, p = 0, depth = 0;
  int C[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  std::vector<double> prm;
  fcm::Geo geo{};
  std::vector<std::vector<uint64_t>> elems;              // per level, sorted
  std::vector<std::unordered_set<uint64_t>> E, R;        // elements, refined
  std::vector<std::unordered_map<uint64_t, long long>> comp;  // active component -> first id
  std::vector<int> f_level, f_t, f_q;                    // per function (t, q: 3 each)
  std::vector<int> leaf_level, leaf_index;               // per leaf (index: 3 each)
  std::vector<signed char> leaf_cls;                     // per leaf: CLS_INSIDE/OUTSIDE/CUT
  int n_levels = 0;                                      // hp-multigrid levels
  std::vector<int> f_coarsest;                           // per function: coarsest level holding it
  std::vector<long long> leaf_off, leaf_fn;
  std::vector<long long> patch_off, patch_fn;

  int lattice(int k, int a) const { return a < dim ? (C[a] << k) : 1; }

  void box(int k, const int* e, double* x0, double* x1) const {
    for (int a = 0; a < 3; ++a) {
      if (a < dim) {
        const double h = (hi[a] - lo[a]) / lattice(k, a);
        x0[a] = lo[a] + e[a] * h;
        x1[a] = lo[a] + (e[a] + 1) * h;
      } else {
        x0[a] = x1[a] = 0.0;
      }
    }
  }

  // In-box lattice cells of level k whose closure contains component t.
  int neighbours(int k, const int* t, uint64_t* out) const {
    int lo_[3], n_[3];
    for (int a = 0; a < 3; ++a) {
      if (a >= dim) {
        lo_[a] = 0;
        n_[a] = 1;
      } else if (t[a] & 1) {
        lo_[a] = (t[a] - 1) / 2;
        n_[a] = 1;
      } else {
        int c0 = t[a] / 2 - 1, c1 = t[a] / 2;
        const int n = lattice(k, a);
        if (c0 < 0) c0 = c1;
        if (c1 >= n) c1 = c0;
        lo_[a] = c0;
        n_[a] = c1 - c0 + 1;
      }
    }
    int cnt = 0;
    for (int z = 0; z < n_[2]; ++z)
      for (int y = 0; y < n_[1]; ++y)
        for (int x = 0; x < n_[0]; ++x) {
          int c[3] = {lo_[0] + x, lo_[1] + y, lo_[2] + z};
          out[cnt++] = pack(c);
        }
    return cnt;
  }

  bool active(int k, const int* t) const {
    uint64_t nb[8];
    const int n = neighbours(k, t, nb);
    const auto& Ek = E[k];
    if (k >= 1)
      for (int i = 0; i < n; ++i)
        if (!Ek.count(nb[i])) return false;  // R1
    bool vertex = true, coarse_vertex = true;
    for (int a = 0; a < dim; ++a) {
      if (t[a] & 1) vertex = false;
      if (t[a] % 4) coarse_vertex = false;
    }
    if (vertex) return !(k >= 1 && coarse_vertex);  // R2
    for (int i = 0; i < n; ++i)
      if (Ek.count(nb[i]) && !R[k].count(nb[i])) return true;  // R3
    return false;
  }

  void build() {
    // elements per level
    E.assign(depth + 1, {});
    R.assign(depth + 1, {});
    elems.assign(depth + 1, {});
    for (int z = 0; z < (dim > 2 ? C[2] : 1); ++z)
      for (int y = 0; y < C[1]; ++y)
        for (int x = 0; x < C[0]; ++x) {
          int e[3] = {x, y, z};
          elems[0].push_back(pack(e));
        }
    E[0].insert(elems[0].begin(), elems[0].end());
    for (int k = 0; k < depth; ++k) {
      for (uint64_t key : elems[k]) {
        int e[3];
        unpack(key, e);
        double x0[3], x1[3];
        box(k, e, x0, x1);
        if (fcm::classify_box(geo, x0, x1) != fcm::CLS_CUT) continue;
        R[k].insert(key);
        for (int oz = 0; oz < (dim > 2 ? 2 : 1); ++oz)
          for (int oy = 0; oy < 2; ++oy)
            for (int ox = 0; ox < 2; ++ox) {
              int c[3] = {2 * e[0] + ox, 2 * e[1] + oy, dim > 2 ? 2 * e[2] + oz : 0};
              E[k + 1].insert(pack(c));
            }
      }
      elems[k + 1].assign(E[k + 1].begin(), E[k + 1].end());
      std::sort(elems[k + 1].begin(), elems[k + 1].end());
    }

    // active components and function numbering
    const int P1 = p + 1, pm = p - 1;
    const int nloc = dim == 3 ? P1 * P1 * P1 : P1 * P1;
    comp.assign(depth + 1, {});
    for (int k = 0; k <= depth; ++k) {
      std::unordered_map<uint64_t, bool> seen;
      std::vector<uint64_t> on;
      for (uint64_t key : elems[k]) {
        int e[3];
        unpack(key, e);
        for (int m = 0; m < nloc; ++m) {
          const int j[3] = {m % P1, (m / P1) % P1, m / (P1 * P1)};
          int t[3] = {0, 0, 0};
          for (int a = 0; a < dim; ++a) t[a] = mode_position(e[a], j[a]);
          const uint64_t tk = pack(t);
          if (seen.count(tk)) continue;
          const bool act = active(k, t);
          seen.emplace(tk, act);
          if (act) on.push_back(tk);
        }
      }
      std::sort(on.begin(), on.end());
      for (uint64_t tk : on) {
        int t[3];
        unpack(tk, t);
        int odd[3], s = 0;
        for (int a = 0; a < dim; ++a)
          if (t[a] & 1) odd[s++] = a;
        long long cnt = 1;
        for (int i = 0; i < s; ++i) cnt *= pm;
        comp[k].emplace(tk, (long long)f_level.size());
        for (long long idx = 0; idx < cnt; ++idx) {
          int q[3] = {0, 0, 0};
          long long r = idx;
          for (int i = 0; i < s; ++i) {
            q[odd[i]] = 2 + (int)(r % pm);
            r /= pm;
          }
          f_level.push_back(k);
          for (int a = 0; a < 3; ++a) {
            f_t.push_back(t[a]);
            f_q.push_back(q[a]);
          }
        }
      }
    }

    // leaves and their functions
    leaf_off.push_back(0);
    for (int k = 0; k <= depth; ++k)
      for (uint64_t key : elems[k]) {
        if (R[k].count(key)) continue;
        int e[3];
        unpack(key, e);
        leaf_level.push_back(k);
        for (int a = 0; a < 3; ++a) leaf_index.push_back(e[a]);
        {
          double x0[3], x1[3];
          box(k, e, x0, x1);
          leaf_cls.push_back((signed char)fcm::classify_box(geo, x0, x1));
        }
        for (int jl = 0; jl <= k; ++jl) {
          int ae[3] = {0, 0, 0};
          for (int a = 0; a < dim; ++a) ae[a] = e[a] >> (k - jl);
          for (int m = 0; m < nloc; ++m) {
            const int j[3] = {m % P1, (m / P1) % P1, m / (P1 * P1)};
            int t[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) t[a] = mode_position(ae[a], j[a]);
            auto it = comp[jl].find(pack(t));
            if (it == comp[jl].end()) continue;
            long long id = it->second, stride = 1;
            for (int a = 0; a < dim; ++a)
              if (t[a] & 1) {
                id += (j[a] - 2) * stride;
                stride *= pm;
              }
            leaf_fn.push_back(id);
          }
        }
        leaf_off.push_back((long long)leaf_fn.size());
      }

    // hp-multigrid levels (Sec. 3.2), coarsest = 0: the degree is lowered
    // first (p, p-1, ..., 1), then at p = 1 the hats of overlay levels K..1
    // are removed, skipping overlay levels without active hats.  A function
    // of degree q >= 2 last appears on the level of degree q; a hat of
    // overlay level k on the levels above the removal of level k.
    {
      std::vector<long long> hats(depth + 1, 0);
      std::vector<int> deg(f_level.size(), 1);
      for (size_t f = 0; f < f_level.size(); ++f) {
        for (int a = 0; a < 3; ++a) deg[f] = std::max(deg[f], f_q[3 * f + a]);
        if (deg[f] == 1) ++hats[f_level[f]];
      }
      std::vector<int> kept;                  // overlay levels whose removal is a level
      for (int kk = depth; kk >= 1; --kk)
        if (hats[kk] > 0) kept.push_back(kk);
      const int nk = (int)kept.size();
      n_levels = p + nk;
      f_coarsest.resize(f_level.size());
      for (size_t f = 0; f < f_level.size(); ++f) {
        if (deg[f] >= 2) {
          f_coarsest[f] = n_levels - 1 - (p - deg[f]);
        } else {
          int above = 0;                      // kept removals of levels above this hat's
          for (int kk : kept) above += kk > f_level[f];
          f_coarsest[f] = n_levels - 1 - (p - 1 + above);
        }
      }
    }

    // patches: functions touching the base cells around each base node
    long long nbase = 1;
    for (int a = 0; a < dim; ++a) nbase *= C[a];
    std::vector<std::vector<long long>> per_cell(nbase);
    for (int k = 0; k <= depth; ++k) {
      std::vector<std::pair<uint64_t, long long>> cs(comp[k].begin(), comp[k].end());
      std::sort(cs.begin(), cs.end(), [](const auto& x, const auto& y) { return x.second < y.second; });
      for (const auto& [tk, first] : cs) {
        int t[3];
        unpack(tk, t);
        long long cnt = 1;
        for (int a = 0; a < dim; ++a)
          if (t[a] & 1) cnt *= pm;
        uint64_t nb[8];
        const int n = neighbours(k, t, nb);
        long long cells[8];
        int nc = 0;
        for (int i = 0; i < n; ++i) {
          if (!E[k].count(nb[i])) continue;
          int c[3];
          unpack(nb[i], c);
          const long long lin = (long long)(c[0] >> k) +
                                (long long)C[0] * ((c[1] >> k) + (long long)C[1] * (c[2] >> k));
          bool dup = false;
          for (int q = 0; q < nc; ++q) dup |= cells[q] == lin;
          if (!dup) cells[nc++] = lin;
        }
        for (int q = 0; q < nc; ++q)
          for (long long f = first; f < first + cnt; ++f) per_cell[cells[q]].push_back(f);
      }
    }
    patch_off.push_back(0);
    const int nz = dim > 2 ? C[2] + 1 : 1;
    std::vector<long long> u;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y <= C[1]; ++y)
        for (int x = 0; x <= C[0]; ++x) {
          u.clear();
          for (int oz = 0; oz < (dim > 2 ? 2 : 1); ++oz)
            for (int oy = 0; oy < 2; ++oy)
              for (int ox = 0; ox < 2; ++ox) {
                const int c[3] = {x - ox, y - oy, dim > 2 ? z - oz : 0};
                bool in = true;
                for (int a = 0; a < dim; ++a) in &= c[a] >= 0 && c[a] < C[a];
                if (!in) continue;
                const auto& lst = per_cell[c[0] + (long long)C[0] * (c[1] + (long long)C[1] * c[2])];
                u.insert(u.end(), lst.begin(), lst.end());
              }
          std::sort(u.begin(), u.end());
          u.erase(std::unique(u.begin(), u.end()), u.end());
          patch_fn.insert(patch_fn.end(), u.begin(), u.end());
          patch_off.push_back((long long)patch_fn.size());
        }
  }
};

namespace {

// Legendre P_0..P_n at x by the three-term recurrence.
void legendre(int n, double x, double* P) {
  P[0] = 1.0;
  if (n >= 1) P[1] = x;
  for (int k = 1; k < n; ++k) P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
}

// Integrated Legendre modes of degree <= p at x (values and derivatives).
void modes_1d(int p, double x, double* N, double* dN) {
  double P[fcm::kMaxP + 1];
  legendre(p, x, P);
  N[0] = 0.5 * (1.0 - x);
  N[1] = 0.5 * (1.0 + x);
  dN[0] = -0.5;
  dN[1] = 0.5;
  for (int j = 2; j <= p; ++j) {
    N[j] = (P[j] - P[j - 2]) / std::sqrt(4.0 * j - 2.0);
    dN[j] = std::sqrt((2.0 * j - 1.0) / 2.0) * P[j - 1];
  }
}

// n-point Gauss-Legendre rule: Newton on P_n from cos(pi (i - 1/4) / (n + 1/2)).
void gauss(int n, double* x, double* w) {
  for (int i = 1; i <= (n + 1) / 2; ++i) {
    double r = std::cos(M_PI * (i - 0.25) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double P[fcm::kMaxP + 2];
      legendre(n, r, P);
      dp = n * (r * P[n] - P[n - 1]) / (r * r - 1.0);
      const double dr = P[n] / dp;
      r -= dr;
      if (std::fabs(dr) <= 1e-17) break;
    }
    double P[fcm::kMaxP + 2];
    legendre(n, r, P);
    dp = n * (r * P[n] - P[n - 1]) / (r * r - 1.0);
    const double wi = 2.0 / ((1.0 - r * r) * dp * dp);
    x[i - 1] = -r;
    w[i - 1] = wi;
    x[n - i] = r;
    w[n - i] = wi;
  }
}

void validate(const fcm_grid* g, const fcm_geometry* geom) {
  if (g->dim != 2 && g->dim != 3) throw Invalid{"fcm_mlhp_create: dim must be 2 or 3"};
  if (g->p < 1 || g->p > fcm::kMaxP) throw Invalid{"fcm_mlhp_create: p outside [1, 8]"};
  if (g->overlay_levels < 0 || g->overlay_levels > kMaxOverlay)
    throw Invalid{"fcm_mlhp_create: overlay_levels outside [0, 10]"};
  if (g->space != FCM_SPACE_TENSOR)
    throw Invalid{"fcm_mlhp_create: the overlay topology is built for tensor-product elements"};
  if (g->overlay_p != 0 && g->overlay_p != g->p)
    throw Invalid{"fcm_mlhp_create: overlays carry the base degree (overlay_p 0 or p)"};
  for (int a = 0; a < g->dim; ++a) {
    if (g->cells[a] < 1) throw Invalid{"fcm_mlhp_create: cells must be >= 1"};
    if (((long long)g->cells[a] << g->overlay_levels) > kMaxLattice)
      throw Invalid{"fcm_mlhp_create: cells * 2^overlay_levels exceeds 2^19 on an axis"};
    if (!std::isfinite(g->lo[a]) || !std::isfinite(g->hi[a]) || !(g->hi[a] > g->lo[a]))
      throw Invalid{"fcm_mlhp_create: box corners must be finite with hi > lo"};
  }
  if (geom->kind < FCM_GEOM_NONE || geom->kind > FCM_GEOM_ELLIPSOID)
    throw Invalid{"fcm_mlhp_create: unknown geometry kind"};
  if (geom->complement != 0 && geom->complement != 1)
    throw Invalid{"fcm_mlhp_create: complement must be 0 or 1"};
  const int need = geom->kind == FCM_GEOM_BALL ? g->dim + 1
                   : geom->kind == FCM_GEOM_ELLIPSOID ? 15
                   : geom->kind == FCM_GEOM_VOIDS ? 4 : 0;
  if (geom->kind == FCM_GEOM_VOIDS && geom->n_params % 4)
    throw Invalid{"fcm_mlhp_create: voids take 4 parameters per ball"};
  if (geom->kind == FCM_GEOM_ELLIPSOID && g->dim != 3)
    throw Invalid{"fcm_mlhp_create: the ellipsoid is 3D"};
  if (geom->n_params < need || (need && !geom->params))
    throw Invalid{"fcm_mlhp_create: too few geometry parameters"};
  for (int i = 0; i < geom->n_params; ++i)
    if (!std::isfinite(geom->params[i]))
      throw Invalid{"fcm_mlhp_create: non-finite geometry parameter"};
}

}  // namespace

extern "C" {

fcm_status fcm_mlhp_create(const fcm_grid* grid, const fcm_geometry* geom, fcm_mlhp** out) {
  if (!out || !grid || !geom) {
    fcm::set_last_error("fcm_mlhp_create: null argument");
    return FCM_E_INVALID;
  }
  *out = nullptr;
  try {
    validate(grid, geom);
    std::unique_ptr<fcm_mlhp> m(new fcm_mlhp());
    m->dim = grid->dim;
    m->p = grid->p;
    m->depth = grid->overlay_levels;
    for (int a = 0; a < 3; ++a) {
      m->C[a] = a < grid->dim ? grid->cells[a] : 1;
      m->lo[a] = grid->lo[a];
      m->hi[a] = grid->hi[a];
    }
    if (geom->n_params > 0) m->prm.assign(geom->params, geom->params + geom->n_params);
    m->geo = fcm::Geo{geom->kind, grid->dim, geom->n_params, m->prm.data(), geom->complement};
    m->build();
    *out = m.release();
    return FCM_OK;
  } catch (const Invalid& e) {
    fcm::set_last_error(e.msg.c_str());
    return FCM_E_INVALID;
  } catch (const std::bad_alloc&) {
    fcm::set_last_error("fcm_mlhp_create: host allocation failed");
    return FCM_E_OOM;
  }
}

void fcm_mlhp_destroy(fcm_mlhp* m) { delete m; }

fcm_status fcm_mlhp_sizes(const fcm_mlhp* m, long long* n_functions, long long* n_leaves,
                          long long* n_leaf_entries, long long* n_patch_entries) {
  if (!m || !n_functions || !n_leaves || !n_leaf_entries || !n_patch_entries) {
    fcm::set_last_error("fcm_mlhp_sizes: null argument");
    return FCM_E_INVALID;
  }
  *n_functions = (long long)m->f_level.size();
  *n_leaves = (long long)m->leaf_level.size();
  *n_leaf_entries = (long long)m->leaf_fn.size();
  *n_patch_entries = (long long)m->patch_fn.size();
  return FCM_OK;
}

fcm_status fcm_mlhp_functions(const fcm_mlhp* m, int* level, int* t, int* q) {
  if (!m || !level || !t || !q) {
    fcm::set_last_error("fcm_mlhp_functions: null argument");
    return FCM_E_INVALID;
  }
  std::copy(m->f_level.begin(), m->f_level.end(), level);
  std::copy(m->f_t.begin(), m->f_t.end(), t);
  std::copy(m->f_q.begin(), m->f_q.end(), q);
  return FCM_OK;
}

fcm_status fcm_mlhp_leaves(const fcm_mlhp* m, int* level, int* index, long long* offsets,
                           long long* functions) {
  if (!m || !level || !index || !offsets || !functions) {
    fcm::set_last_error("fcm_mlhp_leaves: null argument");
    return FCM_E_INVALID;
  }
  std::copy(m->leaf_level.begin(), m->leaf_level.end(), level);
  std::copy(m->leaf_index.begin(), m->leaf_index.end(), index);
  std::copy(m->leaf_off.begin(), m->leaf_off.end(), offsets);
  std::copy(m->leaf_fn.begin(), m->leaf_fn.end(), functions);
  return FCM_OK;
}

fcm_status fcm_mlhp_patches(const fcm_mlhp* m, long long* offsets, long long* functions) {
  if (!m || !offsets || !functions) {
    fcm::set_last_error("fcm_mlhp_patches: null argument");
    return FCM_E_INVALID;
  }
  std::copy(m->patch_off.begin(), m->patch_off.end(), offsets);
  std::copy(m->patch_fn.begin(), m->patch_fn.end(), functions);
  return FCM_OK;
}

fcm_status fcm_mlhp_leaf_classes(const fcm_mlhp* m, signed char* cls) {
  if (!m || !cls) {
    fcm::set_last_error("fcm_mlhp_leaf_classes: null argument");
    return FCM_E_INVALID;
  }
  std::copy(m->leaf_cls.begin(), m->leaf_cls.end(), cls);
  return FCM_OK;
}

fcm_status fcm_mlhp_levels(const fcm_mlhp* m, int* n_levels, int* coarsest) {
  if (!m || !n_levels || !coarsest) {
    fcm::set_last_error("fcm_mlhp_levels: null argument");
    return FCM_E_INVALID;
  }
  *n_levels = m->n_levels;
  std::copy(m->f_coarsest.begin(), m->f_coarsest.end(), coarsest);
  return FCM_OK;
}

fcm_status fcm_mlhp_restriction_1d(int p, int dk, int pos, double* S) {
  if (!S || p < 1 || p > fcm::kMaxP || dk < 0 || dk > kMaxOverlay || pos < 0 || pos >= (1 << dk)) {
    fcm::set_last_error("fcm_mlhp_restriction_1d: invalid argument");
    return FCM_E_INVALID;
  }
  const int P1 = p + 1;
  if (dk == 0) {                                  // the interval itself
    for (int i = 0; i < P1; ++i)
      for (int j = 0; j < P1; ++j) S[i * P1 + j] = i == j ? 1.0 : 0.0;
    return FCM_OK;
  }
  const double s = std::ldexp(1.0, -dk);          // leaf length / ancestor length
  const double c = -1.0 + s * (2 * pos + 1);      // leaf centre in ancestor coordinates
  double N[fcm::kMaxP + 1], dN[fcm::kMaxP + 1];
  // nodal rows: the restricted mode's values at the leaf's end points
  modes_1d(p, c - s, N, dN);
  for (int j = 0; j < P1; ++j) S[j] = N[j];
  modes_1d(p, c + s, N, dN);
  for (int j = 0; j < P1; ++j) S[P1 + j] = N[j];
  // bubble rows: bubble derivatives are orthonormal and orthogonal to the
  // constant derivatives of the nodal modes, so the coefficient of leaf
  // bubble i is int_{-1}^{1} d/dxi [N_j(c + s xi)] N_i'(xi) dxi (Gauss, exact
  // for the degree 2p - 2 integrand with p points).  It vanishes exactly for
  // i > j (the restriction of a degree-j mode has degree j), which includes
  // the nodal columns j = 0, 1.
  double xq[fcm::kMaxP], wq[fcm::kMaxP];
  gauss(p, xq, wq);
  for (int i = 2; i < P1; ++i)
    for (int j = 0; j < P1; ++j) S[i * P1 + j] = 0.0;
  for (int q = 0; q < p; ++q) {
    double Na[fcm::kMaxP + 1], dNa[fcm::kMaxP + 1], Nl[fcm::kMaxP + 1], dNl[fcm::kMaxP + 1];
    modes_1d(p, c + s * xq[q], Na, dNa);
    modes_1d(p, xq[q], Nl, dNl);
    for (int i = 2; i < P1; ++i)
      for (int j = i; j < P1; ++j) S[i * P1 + j] += wq[q] * (s * dNa[j]) * dNl[i];
  }
  return FCM_OK;
}

}  // extern "C"
