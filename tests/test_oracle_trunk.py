"""Pins of the trunk-space oracle (oracle/trunk.py).

* Table tab::upperbound, trunk-space column: the elementwise (n = 1) and
  patchwise (n = 2) block sizes for p = 2..8 and n_f = 1, 3
  (tests/golden/upperbound_trunk_space.json; the p >= 6 row read with the
  factor 1/6 it lacks).
* The global DOF count equals the closed form of vertices, edges, faces and
  interiors of the grid.
* The trunk space reproduces every polynomial of total degree p (L2
  projection exact) and not a Q_p monomial of higher total degree.
* Its p-levels are the trunk spaces of lower degree (direct assembly).
* V-cycle SPD, PCG = direct solve; removing fully fictitious cells removes
  exactly the DOFs they alone support and leaves the physical solution.
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import fcm_inputs as fi
from oracle.assembly import shape_functions
from oracle.geometry import OUTSIDE, levelset
from oracle.grid import all_cells, cell_box, cell_dofs
from oracle.multigrid import pcg
from oracle.quadrature import leaf_rule
from oracle.trunk import (TrunkHierarchy, TrunkSpace, assemble_trunk, trunk_global_mask,
                          trunk_local_mask)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _upperbound(n, p, nf):
    if p < 4:
        return nf * (n + 1) ** 2 * (3 * n * p - 2 * n + 1)
    if p <= 5:
        v = nf * (n + 1) * (3 * n * n * p * p - 9 * n * n * p + 6 * n * p + 14 * n * n - 2 * n + 2)
        assert v % 2 == 0
        return v // 2
    v = nf * (n ** 3 * p ** 3 - 3 * n ** 3 * p ** 2 + 9 * n * n * p * p + 20 * n ** 3 * p
              - 9 * n * n * p + 18 * (n * p - n ** 3 + 2 * n * n) + 6)
    assert v % 6 == 0
    return v // 6


def test_golden_fixture_states_the_formulas():
    with open(os.path.join(GOLDEN, "upperbound_trunk_space.json")) as f:
        g = json.load(f)
    assert set(g["formulas"]) == {"p < 4", "4 <= p <= 5", "p >= 6"}


@pytest.mark.parametrize("p", range(2, 9))
@pytest.mark.parametrize("nf", [1, 3])
def test_trunk_block_sizes_match_upper_bound_table(p, nf):
    # elementwise: the trunk modes of one hexahedron
    assert nf * int(trunk_local_mask(3, p).sum()) == _upperbound(1, p, nf)
    # patchwise: the trunk DOFs of the 2 x 2 x 2 cells around an interior node
    C = (3, 3, 3)
    keep = trunk_global_mask(3, C, p)
    ids = set()
    for c in itertools.product((0, 1), repeat=3):
        ids.update(int(i) for i in cell_dofs(3, C, p, c) if keep[i])
    assert nf * len(ids) == _upperbound(2, p, nf)


@pytest.mark.parametrize("C,p", [((2, 3, 4), 2), ((3, 3, 3), 4), ((2, 2, 3), 6)])
def test_dof_count_closed_form(C, p):
    cx, cy, cz = C
    face = sum(1 for i in range(2, p + 1) for j in range(2, p + 1) if i + j <= p)
    inner = sum(1 for i in range(2, p + 1) for j in range(2, p + 1) for k in range(2, p + 1)
                if i + j + k <= p)
    vertices = (cx + 1) * (cy + 1) * (cz + 1)
    edges = cx * (cy + 1) * (cz + 1) + (cx + 1) * cy * (cz + 1) + (cx + 1) * (cy + 1) * cz
    faces = cx * cy * (cz + 1) + cx * (cy + 1) * cz + (cx + 1) * cy * cz
    expect = vertices + edges * (p - 1) + faces * face + cx * cy * cz * inner
    assert int(trunk_global_mask(3, C, p).sum()) == expect


def _l2_projection_error(p, f, C=(2, 2, 2)):
    prob = dict(fi.poisson3d_sphere(cells=C[0], p=p), cells=C, geometry=dict(kind="none"))
    space = TrunkSpace(prob)
    rows, cols, vals = [], [], []
    b = np.zeros(space.M)
    for c in all_cells(3, C):
        x0, x1 = cell_box(prob["lo"], prob["hi"], C, c)
        pts, w = leaf_rule(x0, x1, p + 1)
        N, _ = shape_functions(p, x0, x1, pts)
        pos, g = space.cell_dofs(c)
        Nt = N[:, pos]
        Me = Nt.T @ (w[:, None] * Nt)
        rows.append(np.repeat(g, len(g)))
        cols.append(np.tile(g, len(g)))
        vals.append(Me.ravel())
        np.add.at(b, g, Nt.T @ (w * f(pts)))
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(space.M, space.M)).tocsc()
    u = spla.spsolve(M, b)
    err = 0.0
    rng = np.random.default_rng(3)
    for c in all_cells(3, C):
        x0, x1 = cell_box(prob["lo"], prob["hi"], C, c)
        pts = np.asarray(x0) + rng.random((20, 3)) * (np.asarray(x1) - np.asarray(x0))
        N, _ = shape_functions(p, x0, x1, pts)
        pos, g = space.cell_dofs(c)
        err = max(err, np.abs(N[:, pos] @ u[g] - f(pts)).max())
    return err


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_reproduces_total_degree_p_and_not_more(p):
    rng = np.random.default_rng(p)
    exps = [e for e in itertools.product(range(p + 1), repeat=3) if sum(e) <= p]
    coef = rng.standard_normal(len(exps))

    def f(x):
        return sum(cf * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c
                   for cf, (a, b, c) in zip(coef, exps))

    assert _l2_projection_error(p, f) < 1e-10
    # x^p y^p is in Q_p (tensor space) but has total degree 2p > p
    assert _l2_projection_error(p, lambda x: x[:, 0] ** p * x[:, 1] ** p) > 1e-6


def _smooth_cube(p):
    return dict(fi.poisson3d_sphere(cells=3, p=p), geometry=dict(kind="none"),
                source=dict(kind="const", f0=1.0),
                dirichlet=dict(kind="faces", g="zero", faces=[0, 3]))


def test_p_levels_are_lower_degree_trunk_spaces():
    prob = _smooth_cube(4)
    H = TrunkHierarchy(prob)
    # levels: h-levels, then p = 1, 2, 3, 4 at the end (finest last)
    p_levels = [lv for lv in H.levels if lv.cells == (3, 3, 3)]
    assert [lv.p for lv in p_levels] == [1, 2, 3, 4]
    for lv in p_levels[:-1]:
        Ad, _, _, _ = assemble_trunk(dict(prob, p=lv.p))
        D = (lv.A - Ad).toarray()
        assert np.abs(D).max() <= 1e-12 * abs(Ad).max(), lv.p


@pytest.fixture(scope="module")
def sphere_trunk():
    return TrunkHierarchy(dict(fi.poisson3d_sphere(cells=4, p=3, radius=0.3), drop_outside=True))


def test_trunk_vcycle_spd_and_pcg(sphere_trunk):
    H = sphere_trunk
    n = H.A.shape[0]
    Vm = np.column_stack([H.vcycle(e) for e in np.eye(n)])
    assert np.abs(Vm - Vm.T).max() <= 1e-8 * np.abs(Vm).max()
    assert np.linalg.eigvalsh(0.5 * (Vm + Vm.T)).min() > 0.0
    xd = spla.spsolve(H.A.tocsc(), H.b)
    x, k, _ = pcg(H.A, H.b, H.vcycle, rtol=1e-12, maxit=200)
    e = x - xd
    assert np.sqrt(e @ (H.A @ e)) / np.sqrt(xd @ (H.A @ xd)) < 1e-9
    assert k <= 40


def test_removing_fictitious_cells():
    prob = fi.poisson3d_sphere(cells=6, p=2, radius=0.3)
    A0, b0, s0, classes = assemble_trunk(prob)
    A1, b1, s1, _ = assemble_trunk(dict(prob, drop_outside=True))
    assert (classes == OUTSIDE).sum() > 0
    # the kept DOFs are exactly those touching a cell that is not outside
    touch = set()
    for c, k in zip(all_cells(3, prob["cells"]), classes):
        if k != OUTSIDE:
            touch.update(int(i) for i in cell_dofs(3, prob["cells"], 2, c))
    assert set(s1.tensor_index.tolist()) == touch & set(s0.tensor_index.tolist())
    assert s1.M < s0.M
    # the field in the physical domain barely changes (the removed cells only
    # carried alpha = 1e-8 stiffness); coefficients of DOFs that the
    # fictitious part controls may move, the physical field may not
    x0 = spla.spsolve(A0.tocsc(), b0)
    x1 = spla.spsolve(A1.tocsc(), b1)
    rng = np.random.default_rng(0)
    err = scale = 0.0
    for c, k in zip(all_cells(3, prob["cells"]), classes):
        if k == OUTSIDE:
            continue
        lo, hi = (np.asarray(v) for v in cell_box(prob["lo"], prob["hi"], prob["cells"], c))
        pts = lo + rng.random((30, 3)) * (hi - lo)
        pts = pts[levelset(prob["geometry"], pts) <= 0.0]
        if not len(pts):
            continue
        N, _ = shape_functions(2, lo, hi, pts)
        (p0, g0), (p1, g1) = s0.cell_dofs(c), s1.cell_dofs(c)
        u1 = N[:, p1] @ x1[g1]
        err = max(err, np.abs(N[:, p0] @ x0[g0] - u1).max())
        scale = max(scale, np.abs(u1).max())
    assert err <= 1e-5 * scale
