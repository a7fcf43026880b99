"""Level-set geometry and cell classification (oracle).

Test infrastructure only (see ``oracle/__init__``).

FCM embeds the physical domain in a box and marks it by an indicator alpha
(Sec. 2.1, Eq. weakform): alpha = 1 in Omega_phys, alpha = eps << 1 in
Omega_fict.  Geometry is given by a level set psi with Omega_phys = {psi <= 0}
(the popcorn convention of Sec. 4.3.2, points on the surface count as
physical).

Kinds:
  none       psi = -1 everywhere (body-fitted box)
  ball       psi = |x - c| - r                         (circle / sphere)
  voids      psi = max_k (r_k - |x - c_k|)             (block minus balls)
  ellipsoid  psi = |diag(1/a) R^T (x - c)| - 1
  popcorn    psi = |x| - r0 - sum_k A exp(-|x - c_k|^2 / sigma^2)   (Sec. 4.3.2)
  rotated_square  psi = max(|x'|, |y'|) - a, (x', y') = R(-psi_angle)(x - c)
                  (the rotated square of Sec. 4.1.2)

complement (optional, default False): the physical domain is the other
side, Omega_phys = {psi >= 0} (a hole instead of an inclusion; the paper's
level sets mark either side, e.g. the voids of Sec. 4.3 are fictitious
balls).  The reading: psi is negated exactly, and the box classification
swaps INSIDE and OUTSIDE (CUT stays), so the space-tree quadrature visits
the same cut cells and leaves with the indicator alpha swapped.

Box classification (the paper leaves the cut test open; this is the
reading): balls and voids use exact nearest/farthest point distances, the
ellipsoid and the popcorn a sign test of psi on a 5^d lattice including the
corners (``classify_grid`` evaluates the same test for a whole grid at once,
with the same arithmetic).
Floating-point operations are written out in a fixed order so that a second
implementation performing the same operations gets identical results.
"""
from __future__ import annotations

import numpy as np

INSIDE, OUTSIDE, CUT = 0, 1, 2


def levelset(geom: dict, x: np.ndarray) -> np.ndarray:
    """psi at points x of shape (..., d) (negated for a complement domain)."""
    v = _levelset_kind(geom, x)
    return -v if geom.get("complement") else v


def _swap(cls):
    """INSIDE <-> OUTSIDE, CUT kept (a class or an array of classes)."""
    if np.ndim(cls) == 0:
        return OUTSIDE if cls == INSIDE else (INSIDE if cls == OUTSIDE else cls)
    out = cls.copy()
    out[cls == INSIDE] = OUTSIDE
    out[cls == OUTSIDE] = INSIDE
    return out


def _levelset_kind(geom: dict, x: np.ndarray) -> np.ndarray:
    """psi of the geometry kind at points x of shape (..., d)."""
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[-1]
    kind = geom["kind"]
    if kind == "none":
        return -np.ones(x.shape[:-1])
    if kind == "ball":
        c = geom["center"]
        s = (x[..., 0] - c[0]) * (x[..., 0] - c[0])
        for a in range(1, d):
            s = s + (x[..., a] - c[a]) * (x[..., a] - c[a])
        return np.sqrt(s) - geom["radius"]
    if kind == "voids":
        out = None
        for (cx, cy, cz, r) in geom["balls"]:
            c = (cx, cy, cz)
            s = (x[..., 0] - c[0]) * (x[..., 0] - c[0])
            for a in range(1, d):
                s = s + (x[..., a] - c[a]) * (x[..., a] - c[a])
            v = r - np.sqrt(s)
            out = v if out is None else np.maximum(out, v)
        return out
    if kind == "ellipsoid":
        c, ax, R = geom["center"], geom["axes"], geom["rot"]
        dx = [x[..., a] - c[a] for a in range(3)]
        q = None
        for i in range(3):
            y = R[0][i] * dx[0] + R[1][i] * dx[1] + R[2][i] * dx[2]
            t = y / ax[i]
            q = t * t if q is None else q + t * t
        return np.sqrt(q) - 1.0
    if kind == "rotated_square":
        xp, yp = rotated_coordinates(geom["center"], geom["angle"], x)
        return np.maximum(np.abs(xp), np.abs(yp)) - geom["half"]
    if kind == "popcorn":
        r0, amp, sig2 = geom["r0"], geom["A"], geom["sigma"] * geom["sigma"]
        s = x[..., 0] * x[..., 0] + x[..., 1] * x[..., 1] + x[..., 2] * x[..., 2]
        out = np.sqrt(s) - r0
        for (cx, cy, cz) in geom["centers"]:
            d2 = ((x[..., 0] - cx) * (x[..., 0] - cx) + (x[..., 1] - cy) * (x[..., 1] - cy)
                  + (x[..., 2] - cz) * (x[..., 2] - cz))
            out = out - amp * np.exp(-d2 / sig2)
        return out
    raise ValueError(kind)


def rotated_coordinates(center, angle, x):
    """Coordinates of 2D points x in the frame centred at `center` and
    rotated by `angle` (radians): x' = cos dx + sin dy, y' = -sin dx + cos dy."""
    c, s = np.cos(angle), np.sin(angle)
    dx = x[..., 0] - center[0]
    dy = x[..., 1] - center[1]
    return c * dx + s * dy, -s * dx + c * dy


def _ball_dist2(lo, hi, c):
    """(nearest, farthest) squared distance from c to the box [lo, hi]."""
    dmin2 = 0.0
    dmax2 = 0.0
    for a in range(len(lo)):
        l = lo[a] - c[a]
        u = hi[a] - c[a]
        near = 0.0
        if l > 0.0:
            near = l
        elif u < 0.0:
            near = -u
        far = max(abs(l), abs(u))
        dmin2 = dmin2 + near * near
        dmax2 = dmax2 + far * far
    return dmin2, dmax2


def classify_box(geom: dict, lo, hi) -> int:
    """INSIDE (all physical), OUTSIDE (all fictitious) or CUT."""
    c = _classify_box_kind(geom, lo, hi)
    return _swap(c) if geom.get("complement") else c


def _classify_box_kind(geom: dict, lo, hi) -> int:
    """classify_box for the kind's own domain {psi <= 0}."""
    kind = geom["kind"]
    if kind == "none":
        return INSIDE
    if kind == "ball":
        r = geom["radius"]
        dmin2, dmax2 = _ball_dist2(lo, hi, geom["center"])
        r2 = r * r
        if dmax2 <= r2:
            return INSIDE
        if dmin2 >= r2:
            return OUTSIDE
        return CUT
    if kind == "voids":
        all_clear = True
        for (cx, cy, cz, r) in geom["balls"]:
            dmin2, dmax2 = _ball_dist2(lo, hi, (cx, cy, cz))
            r2 = r * r
            if dmax2 <= r2:
                return OUTSIDE
            if dmin2 < r2:
                all_clear = False
        return INSIDE if all_clear else CUT
    if kind in ("ellipsoid", "popcorn", "rotated_square"):
        d = len(lo)
        ts = [k * 0.25 for k in range(5)]
        pts = []
        for kz in range(5):
            for ky in range(5):
                for kx in range(5):
                    k = (kx, ky, kz)
                    pts.append([lo[a] + ts[k[a]] * (hi[a] - lo[a]) for a in range(d)])
        psi = _levelset_kind(geom, np.array(pts))
        if np.all(psi <= 0.0):
            return INSIDE
        if np.all(psi > 0.0):
            return OUTSIDE
        return CUT
    raise ValueError(kind)


def _classify_grid_voids(geom, lo, hi, cells):
    """The voids test of ``classify_box`` for every cell of a 3D grid at
    once (same per-axis arithmetic)."""
    shape = (cells[2], cells[1], cells[0])
    x0, x1 = [], []
    for a in range(3):
        h = (hi[a] - lo[a]) / cells[a]
        c = np.arange(cells[a], dtype=np.float64)
        x0.append(lo[a] + c * h)
        x1.append(lo[a] + (c + 1.0) * h)
    bcast = [(None, None, slice(None)), (None, slice(None), None), (slice(None), None, None)]
    outside = np.zeros(shape, dtype=bool)
    clear = np.ones(shape, dtype=bool)
    for (cx, cy, cz, r) in geom["balls"]:
        c = (cx, cy, cz)
        dmin2 = np.zeros(shape)
        dmax2 = np.zeros(shape)
        for a in range(3):
            l = x0[a] - c[a]
            u = x1[a] - c[a]
            near = np.where(l > 0.0, l, np.where(u < 0.0, -u, 0.0))
            far = np.maximum(np.abs(l), np.abs(u))
            dmin2 = dmin2 + (near * near)[bcast[a]]
            dmax2 = dmax2 + (far * far)[bcast[a]]
        r2 = r * r
        outside |= dmax2 <= r2
        clear &= ~(dmin2 < r2)
    cls = np.full(shape, CUT, dtype=np.int8)
    cls[clear] = INSIDE
    cls[outside] = OUTSIDE
    return cls.ravel()


def classify_grid(geom: dict, lo, hi, cells) -> np.ndarray:
    """Classes of all cells of a 3D grid (see _classify_grid_kind), swapped
    for a complement domain."""
    c = _classify_grid_kind(geom, lo, hi, cells)
    return _swap(c) if geom.get("complement") else c


def _classify_grid_kind(geom: dict, lo, hi, cells) -> np.ndarray:
    """Classes of all cells of a 3D grid (linear order, x fastest): the test
    of ``classify_box`` evaluated for every cell at once.  Lattice-tested
    kinds use the lattice points lo_c + t (hi_c - lo_c) with the cell corners
    lo_c = lo + c h, hi_c = lo + (c + 1) h, h = (hi - lo) / C."""
    if geom["kind"] == "voids":
        return _classify_grid_voids(geom, lo, hi, cells)
    assert geom["kind"] in ("ellipsoid", "popcorn") and len(cells) == 3
    ts = [k * 0.25 for k in range(5)]
    axes = []
    for a in range(3):
        h = (hi[a] - lo[a]) / cells[a]
        c = np.arange(cells[a], dtype=np.float64)
        x0 = lo[a] + c * h
        x1 = lo[a] + (c + 1.0) * h
        axes.append([x0 + t * (x1 - x0) for t in ts])
    shape = (cells[2], cells[1], cells[0])
    any_in = np.zeros(shape, dtype=bool)
    any_out = np.zeros(shape, dtype=bool)
    for kz in range(5):
        for ky in range(5):
            for kx in range(5):
                X = np.empty(shape + (3,))
                X[..., 0] = axes[0][kx][None, None, :]
                X[..., 1] = axes[1][ky][None, :, None]
                X[..., 2] = axes[2][kz][:, None, None]
                v = _levelset_kind(geom, X)
                any_in |= v <= 0.0
                any_out |= v > 0.0
    cls = np.full(shape, CUT, dtype=np.int8)
    cls[~any_out] = INSIDE
    cls[~any_in] = OUTSIDE
    return cls.ravel()
