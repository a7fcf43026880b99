"""Pins of the cube with spherical cavities (Sec. 4.3) in the oracle: the
paper's DOF counts for trunk-space elasticity with the fictitious cells
removed, on uniform grids (h = 1/32, p = 2 and h = 1/128, p = 5) and on the
overlay meshes of its refinement study (k = 1, 2), and its CG+MG iteration
range, under the geometry reading of tests/golden/cube_cavities_dofs.json.
The whole-grid voids cut test equals the per-cell one."""
import json
import os

import fcm_inputs as fi
from oracle.geometry import classify_box, classify_grid
from oracle.grid import all_cells, cell_box
from oracle.mlhp import MlhpSpace, kept_functions, mesh_for
from oracle.multigrid import pcg
from oracle.trunk import TrunkHierarchy, TrunkSpace

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    with open(os.path.join(GOLDEN, "cube_cavities_dofs.json")) as f:
        return json.load(f)


def test_classify_grid_voids_is_the_cell_test():
    prob = dict(fi.cube_cavities(), cells=(7, 9, 11))
    got = classify_grid(prob["geometry"], prob["lo"], prob["hi"], prob["cells"])
    ref = [classify_box(prob["geometry"], *cell_box(prob["lo"], prob["hi"], prob["cells"], c))
           for c in all_cells(3, prob["cells"])]
    assert got.tolist() == ref


def test_uniform_dof_counts():
    g = _golden()
    for case in g["uniform"]:
        prob = fi.cube_cavities(cells=case["cells"], p=case["p"])
        cls = classify_grid(prob["geometry"], prob["lo"], prob["hi"], prob["cells"])
        n = 3 * TrunkSpace(prob, cls).M
        assert abs(n - case["dofs"]) <= g["tolerance_uniform"] * case["dofs"], (case, n)


def test_overlay_dof_counts():
    g = _golden()
    ov = g["overlays"]
    for k, ref in zip(ov["k"], ov["dofs"]):
        prob = fi.cube_cavities(cells=ov["cells"], p=ov["p"], overlay_levels=k)
        space = MlhpSpace(mesh_for(prob), ov["p"], nf=1, trunk=True)
        n = 3 * int(kept_functions(space, prob["geometry"]).sum())
        assert abs(n - ref) <= g["tolerance_overlays"] * ref, (k, n)


def test_iterations_in_the_papers_range():
    """Sec. 4.3: 16-19 CG+MG iterations at p = 2 for h = 1/32..1/128,
    independent of h.  The oracle needs 14, 18, 15 and 15 at h = 1/8,
    1/12, 1/16 and 1/32 (and 13 at h = 1/16, p = 3, paper 14-15); its coarse
    solver differs from the paper's.  Checked at h = 1/12, a cheap grid on
    which a cavity still spans several cells.  Bar: within 2 of the printed
    range."""
    lo, hi = _golden()["iterations"]["p2"]
    H = TrunkHierarchy(fi.cube_cavities(cells=12, p=2))
    _, k, _ = pcg(H.A, H.b, H.vcycle, rtol=1e-9, maxit=200)
    assert lo - 2 <= k <= hi + 2, k
