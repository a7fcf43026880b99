"""Cut-cell and boundary quadrature (oracle).

Test infrastructure only (see ``oracle/__init__``).

Volume integrals on cut cells use a space tree (Sec. 2.1 and the rod example
of Sec. 4.3.1, "octree ... depth of 3"): a cut (sub)cell is bisected along
every axis until it is uncut or the maximum depth is reached.  Each leaf gets
a (p+1)^d Gauss-Legendre rule.  Uncut leaves carry the constant alpha of
their class; leaves still cut at the maximum depth evaluate alpha point by
point (psi <= 0 -> 1, else the fictitious factor).  The paper does not state
the number of points per leaf or the cut test; (p+1)^d points and the tests
of ``geometry.classify_box`` are the readings.

Dirichlet data on the immersed boundary are imposed by penalty (Eq. weakform,
second integral).  The paper extracts the surface with marching cubes
(Sec. 4.3.2); the reading here is marching simplices on every leaf that is
still cut at the maximum depth: the leaf is split into the d! Kuhn simplices
that share its main diagonal, psi is interpolated linearly along each edge
whose end values change sign (psi <= 0 counts as inside), and the zero set of
each simplex is a segment (2D), a triangle, or a quadrilateral split into two
triangles (3D).  Segments get a (p+1)-point Gauss rule, triangles a
collapsed (Duffy) product of two (p+1)-point rules.
"""
from __future__ import annotations

import functools
import itertools
import math

import numpy as np

from .basis import gauss_legendre
from .geometry import CUT, INSIDE, classify_box, levelset


@functools.lru_cache(maxsize=None)
def _reference_tensor_rule(n, d):
    """Reference nodes (Q, d) and per-axis weights (Q, d), x fastest."""
    xi, wi = gauss_legendre(n)
    idx = np.array([t[::-1] for t in itertools.product(*[range(n)] * d)])
    return xi[idx], wi[idx]


def leaf_rule(lo, hi, p):
    """Tensor (p+1)^d Gauss rule on the box [lo, hi] (x fastest):
    x = (lo+hi)/2 + (hi-lo)/2 * xi, w = prod_a (hi_a-lo_a)/2 * w_a."""
    d = len(lo)
    XI, WI = _reference_tensor_rule(p + 1, d)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    mids = 0.5 * (lo + hi)
    hds = 0.5 * (hi - lo)
    pts = mids + hds * XI
    hw = hds * WI
    w = hw[:, 0]
    for a in range(1, d):
        w = w * hw[:, a]
    return pts, w


def kuhn_simplices(d):
    """Vertex-id sequences of the d! Kuhn simplices of a box (corner id bit a
    set = upper end along axis a)."""
    out = []
    for perm in itertools.permutations(range(d)):
        k = 0
        seq = [k]
        for a in perm:
            k = k | (1 << a)
            seq.append(k)
        out.append(seq)
    return out


def _edge_point(v, psi, i, j):
    t = psi[i] / (psi[i] - psi[j])
    return v[i] + t * (v[j] - v[i])


def marching_simplices(lo, hi, psi_fn):
    """Zero-set pieces of the linear interpolant of psi on the Kuhn
    simplices of the box.  Returns a list of point tuples: 2 points per
    segment (2D) or 3 per triangle (3D)."""
    d = len(lo)
    corners = []
    for k in range(1 << d):
        corners.append([hi[a] if (k >> a) & 1 else lo[a] for a in range(d)])
    corners = np.array(corners)
    psi = psi_fn(corners)
    pieces = []
    for seq in kuhn_simplices(d):
        ins = [i for i in seq if psi[i] <= 0.0]
        out = [j for j in seq if psi[j] > 0.0]
        if not ins or not out:
            continue
        if d == 2:
            if len(ins) == 1:
                i = ins[0]
                pieces.append((_edge_point(corners, psi, i, out[0]),
                               _edge_point(corners, psi, i, out[1])))
            else:
                j = out[0]
                pieces.append((_edge_point(corners, psi, ins[0], j),
                               _edge_point(corners, psi, ins[1], j)))
        else:
            if len(ins) == 1:
                i = ins[0]
                pieces.append(tuple(_edge_point(corners, psi, i, j) for j in out))
            elif len(ins) == 3:
                j = out[0]
                pieces.append(tuple(_edge_point(corners, psi, i, j) for i in ins))
            else:
                i1, i2 = ins
                j1, j2 = out
                q0 = _edge_point(corners, psi, i1, j1)
                q1 = _edge_point(corners, psi, i1, j2)
                q2 = _edge_point(corners, psi, i2, j2)
                q3 = _edge_point(corners, psi, i2, j1)
                pieces.append((q0, q1, q2))
                pieces.append((q0, q2, q3))
    return pieces


def piece_rule(piece, p):
    """Gauss rule on a segment (2 points) or a triangle (3 points)."""
    xi, wi = gauss_legendre(p + 1)
    u = 0.5 * (xi + 1.0)
    wu = 0.5 * wi
    if len(piece) == 2:
        A, B = piece
        L = math.sqrt(float(np.sum((B - A) * (B - A))))
        return A + u[:, None] * (B - A), wu * L
    A, B, C = piece
    e1 = B - A
    e2 = C - B
    cr = np.array([e1[1] * e2[2] - e1[2] * e2[1],
                   e1[2] * e2[0] - e1[0] * e2[2],
                   e1[0] * e2[1] - e1[1] * e2[0]])
    J = math.sqrt(float(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]))
    ui = np.repeat(u, p + 1)
    uj = np.tile(u, p + 1)
    pts = A + ui[:, None] * e1 + (ui * uj)[:, None] * e2
    wts = np.repeat(wu, p + 1) * np.tile(wu, p + 1) * ui * J
    return pts, wts


def cell_rules(prob, x0, x1, cls=None):
    """Volume and immersed-surface rules of one cell.

    Returns (vol_pts, vol_w, vol_alpha, surf_pts, surf_w); the surface part
    is empty unless Dirichlet data live on the level set."""
    geom = prob["geometry"]
    p = prob["p"]
    depth = prob["quad_depth"]
    afict = prob["alpha"]
    want_surf = prob["dirichlet"]["kind"] == "levelset"
    d = len(x0)
    vp, vw, va, sp, sw = [], [], [], [], []

    def psi_fn(x):
        return levelset(geom, x)

    def rec(lo, hi, level):
        c = classify_box(geom, lo, hi)
        if c != CUT:
            pts, wts = leaf_rule(lo, hi, p)
            vp.append(pts)
            vw.append(wts)
            va.append(np.full(len(wts), 1.0 if c == INSIDE else afict))
            return
        if level == depth:
            pts, wts = leaf_rule(lo, hi, p)
            psi = psi_fn(pts)
            vp.append(pts)
            vw.append(wts)
            va.append(np.where(psi <= 0.0, 1.0, afict))
            if want_surf:
                for piece in marching_simplices(lo, hi, psi_fn):
                    spts, swts = piece_rule(piece, p)
                    sp.append(spts)
                    sw.append(swts)
            return
        mid = [0.5 * (lo[a] + hi[a]) for a in range(d)]
        for k in range(1 << d):
            clo = [mid[a] if (k >> a) & 1 else lo[a] for a in range(d)]
            chi = [hi[a] if (k >> a) & 1 else mid[a] for a in range(d)]
            rec(clo, chi, level + 1)

    rec(list(x0), list(x1), 0)
    vol = (np.concatenate(vp), np.concatenate(vw), np.concatenate(va))
    if sp:
        surf = (np.concatenate(sp), np.concatenate(sw))
    else:
        surf = (np.zeros((0, d)), np.zeros(0))
    return vol + surf


def face_rule(x0, x1, face, p):
    """(p+1)^(d-1) Gauss rule on face `face` = 2 a + s of the box [x0, x1]
    (a = normal axis, s = 0 lower / 1 upper side)."""
    d = len(x0)
    a = face // 2
    s = face % 2
    xi, wi = gauss_legendre(p + 1)
    others = [b for b in range(d) if b != a]
    pts, wts = [], []
    for idx in itertools.product(*[range(p + 1)] * (d - 1)):
        idx = idx[::-1]
        x = [0.0] * d
        x[a] = x1[a] if s else x0[a]
        w = 1.0
        for k, b in enumerate(others):
            mid = 0.5 * (x0[b] + x1[b])
            hd = 0.5 * (x1[b] - x0[b])
            x[b] = mid + hd * xi[idx[k]]
            w = w * (hd * wi[idx[k]])
        pts.append(x)
        wts.append(w)
    return np.array(pts), np.array(wts)
