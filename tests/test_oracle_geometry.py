"""Pins of the oracle's geometry and cut-cell quadrature.

Cell classes are checked against dense point sampling; the space-tree volume
rule against the exact area / volume of circles, spheres and ellipsoids; the
marching-simplex surface rule against exact perimeters and areas."""
import math

import numpy as np
import pytest

import fcm_inputs as fi
from oracle.geometry import CUT, INSIDE, OUTSIDE, classify_box, levelset
from oracle.grid import all_cells, cell_box
from oracle.quadrature import cell_rules, leaf_rule


GEOMS = [
    dict(kind="ball", center=(0.5, 0.5, 0.5), radius=0.45),
    dict(kind="voids", balls=[[0.3, 0.4, 0.5, 0.12], [0.7, 0.6, 0.4, 0.08]]),
    dict(kind="ellipsoid", center=(0.5, 0.5, 0.5), axes=(0.4, 0.25, 0.3),
         rot=fi.random_rotation(fi.SplitMix64(7))),
]


@pytest.mark.parametrize("geom", GEOMS)
def test_classification_agrees_with_sampling(geom):
    rng = np.random.default_rng(3)
    for _ in range(300):
        lo = rng.uniform(0, 0.9, 3)
        hi = lo + rng.uniform(0.01, 0.2, 3)
        c = classify_box(geom, lo, hi)
        pts = lo + (hi - lo) * rng.uniform(0, 1, (400, 3))
        psi = levelset(geom, pts)
        if c == INSIDE:
            assert np.all(psi <= 1e-12)
        elif c == OUTSIDE:
            assert np.all(psi > -1e-12)
        elif geom["kind"] == "ball":
            # exact test: the box's nearest and farthest points straddle r
            cc = np.array(geom["center"])
            near = np.clip(cc, lo, hi)
            far = np.where(np.abs(lo - cc) > np.abs(hi - cc), lo, hi)
            assert levelset(geom, near[None])[0] < 1e-12
            assert levelset(geom, far[None])[0] > -1e-12


def _measure(prob, surf=False):
    vol = 0.0
    area = 0.0
    for cell in all_cells(prob["dim"], prob["cells"]):
        x0, x1 = cell_box(prob["lo"], prob["hi"], prob["cells"], cell)
        c = classify_box(prob["geometry"], x0, x1)
        if c == CUT:
            vp, vw, va, sp_, sw = cell_rules(prob, x0, x1)
            vol += float(np.sum(vw[va == 1.0]))
            area += float(np.sum(sw))
        elif c == INSIDE:
            _, w = leaf_rule(x0, x1, prob["p"])
            vol += float(np.sum(w))
    return vol, area


@pytest.mark.parametrize("depth,tol", [(1, 1.5e-2), (3, 2e-3), (5, 3e-4)])
def test_circle_area_and_perimeter(depth, tol):
    r = 0.4
    prob = fi.poisson2d_circle(cells=8, p=2, radius=r, quad_depth=depth)
    vol, per = _measure(prob)
    assert abs(vol - math.pi * r * r) / (math.pi * r * r) < tol
    assert abs(per - 2 * math.pi * r) / (2 * math.pi * r) < tol


def test_sphere_volume_and_area():
    r = 0.45
    prob = fi.poisson3d_sphere(cells=4, p=1, radius=r, quad_depth=3)
    vol, area = _measure(prob)
    assert abs(vol - 4 / 3 * math.pi * r ** 3) / (4 / 3 * math.pi * r ** 3) < 5e-3
    assert abs(area - 4 * math.pi * r * r) / (4 * math.pi * r * r) < 5e-3


def test_area_converges_under_tree_depth():
    r = 0.4
    errs = []
    for depth in (1, 2, 3, 4):
        prob = fi.poisson2d_circle(cells=4, p=1, radius=r, quad_depth=depth)
        _, per = _measure(prob)
        errs.append(abs(per - 2 * math.pi * r))
    # linear interpolation of a smooth curve: error ~ leaf size^2
    assert errs[-1] < errs[0] / 20


def test_ellipsoid_volume():
    g = GEOMS[2]
    prob = fi.poisson3d_sphere(cells=4, p=1, quad_depth=3)
    prob["geometry"] = g
    vol, _ = _measure(prob)
    exact = 4 / 3 * math.pi * np.prod(g["axes"])
    assert abs(vol - exact) / exact < 1e-2


def test_void_sampler_respects_gaps():
    v = fi.draw_voids(64, seed=0, gap=1 / 64)
    assert v.shape == (64, 4)
    assert np.all(v[:, 3] >= 0.03) and np.all(v[:, 3] <= 0.08)
    for i in range(64):
        c, r = v[i, :3], v[i, 3]
        assert np.all(c - r >= 1 / 64 - 1e-15) and np.all(c + r <= 1 - 1 / 64 + 1e-15)
        for j in range(i):
            assert np.linalg.norm(c - v[j, :3]) >= r + v[j, 3] + 1 / 64 - 1e-12


# Complement domains (the geometry's "complement" flag, Omega_phys = {psi >= 0}).

@pytest.mark.parametrize("geom", GEOMS)
def test_complement_classification_agrees_with_sampling(geom):
    """A complement box class holds for sampled points of the complement:
    INSIDE boxes lie in {psi >= 0}, OUTSIDE boxes in {psi < 0}."""
    gc = dict(geom, complement=True)
    rng = np.random.default_rng(4)
    seen = set()
    for _ in range(300):
        lo = rng.uniform(0, 0.9, 3)
        hi = lo + rng.uniform(0.01, 0.2, 3)
        c = classify_box(gc, lo, hi)
        seen.add(c)
        pts = lo + (hi - lo) * rng.uniform(0, 1, (400, 3))
        psi_kind = levelset(geom, pts)
        assert np.array_equal(levelset(gc, pts), -psi_kind)
        if c == INSIDE:
            assert np.all(psi_kind >= -1e-12)
        elif c == OUTSIDE:
            assert np.all(psi_kind < 1e-12)
    assert CUT in seen and len(seen) == (2 if geom["kind"] == "voids" else 3)


def test_complement_circle_area_and_perimeter():
    """The square with a circular hole: area 1 - pi r^2, the same perimeter."""
    r = 0.4
    prob = fi.poisson2d_circle(cells=8, p=2, radius=r, quad_depth=5)
    prob["geometry"] = dict(prob["geometry"], complement=True)
    vol, per = _measure(prob)
    area = 1.0 - math.pi * r * r
    assert abs(vol - area) / area < 3e-4 * math.pi * r * r / area
    assert abs(per - 2 * math.pi * r) / (2 * math.pi * r) < 3e-4


@pytest.mark.parametrize("pde", ["poisson", "elasticity"])
def test_complement_cell_matrices_sum_to_the_uncut_ones(pde):
    """alpha_Omega + alpha_complement = 1 + alpha pointwise, and both sides
    use the same space tree, so on every cell K(Omega) + K(complement) =
    (1 + alpha) K(uncut), with the penalty terms of the shared surface
    counted twice; checked without the penalty (beta = 0) to 1e-12
    relative, cut cells included."""
    from oracle.assembly import element_system
    if pde == "poisson":
        prob = fi.poisson3d_sphere(cells=4, p=2, radius=0.35, quad_depth=2)
    else:
        prob = fi.elasticity3d_voids(cells=4, p=1, n_voids=3, seed=1)
        prob["quad_depth"] = 2
    prob = dict(prob, beta=0.0)
    comp = dict(prob, geometry=dict(prob["geometry"], complement=True))
    box = dict(prob, geometry=dict(kind="none"))
    ncut = 0
    for cell in all_cells(prob["dim"], prob["cells"]):
        K1, _, c1 = element_system(prob, cell)
        K2, _, c2 = element_system(comp, cell)
        K0, _, _ = element_system(box, cell)
        ncut += c1 == CUT
        assert (c1 == CUT) == (c2 == CUT) and (c1 == INSIDE) == (c2 == OUTSIDE)
        ref = (1.0 + prob["alpha"]) * K0
        assert np.abs(K1 + K2 - ref).max() <= 1e-12 * np.abs(ref).max(), cell
    assert ncut > 0
