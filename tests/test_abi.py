"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/fcm.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fcm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fcm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fcm_setup", "fcm_vcycle", "fcm_pcg_solve", "fcm_apply", "fcm_destroy",
              "fcm_last_error", "fcm_pcg_solve_host"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2010_00881_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_2010_00881_gb300 import fcm
    assert sorted(fcm.EXPORTS) == declared_functions()


def test_last_error_without_gpu():
    from paper_2010_00881_gb300 import fcm
    lib = fcm.load()
    assert lib.fcm_ndofs(None, None) == fcm.FCM_E_INVALID
    assert b"null" in lib.fcm_last_error()


def test_descriptor_marshalling_roundtrip():
    import fcm_inputs as fi
    from paper_2010_00881_gb300 import fcm
    prob = fi.poisson3d_sphere(cells=32, p=3)
    g, gm, ph, op, keep = fcm.descriptors(prob)
    assert (g.dim, tuple(g.cells), g.p) == (3, (32, 32, 32), 3)
    assert gm.kind == fcm.GEOM["ball"] and gm.n_params == 4
    assert [gm.params[i] for i in range(4)] == [0.5, 0.5, 0.5, 0.45]
    assert ph.alpha == 1e-8 and ph.beta == 1e4 and ph.dirichlet == fcm.DIR["levelset"]
    assert (op.n_pre, op.n_post, op.coarse_cells) == (5, 5, 4)
    prob = fi.square_mms(cells=8, p=2)
    g, gm, ph, op, keep = fcm.descriptors(prob)
    assert ph.dirichlet_faces == 0b1111 and ph.kappa == 10.0


def test_dof_layout_matches_the_oracle():
    """fcm_dof_layout / fcm_cell_dofs (host functions, no GPU) against the
    oracle's numbering of the hierarchical basis, bit-exact."""
    from oracle.grid import all_cells, cell_dofs as ocell, dof_1d
    from paper_2010_00881_gb300 import fcm
    for C_, p in ((1, 1), (5, 3), (8, 4)):
        m = fcm.dof_layout(C_, p)
        assert [[dof_1d(C_, c, j) for j in range(p + 1)] for c in range(C_)] == m.tolist()
    for dim, cells, p, nf in (((2, (3, 4), 2, 1)), (3, (2, 3, 2), 3, 1), (3, (3, 2, 2), 2, 3),
                              (2, (5, 1), 1, 2)):
        for lin, cell in enumerate(all_cells(dim, cells)):
            got = fcm.cell_dofs(dim, cells, p, nf, lin)
            assert got.tolist() == ocell(dim, cells, p, cell, nf).tolist(), (dim, cells, p, cell)


def test_dof_layout_rejects_invalid_input():
    from paper_2010_00881_gb300 import fcm
    import pytest as _pytest
    with _pytest.raises(fcm.FcmError):
        fcm.dof_layout(0, 2)
    with _pytest.raises(fcm.FcmError):
        fcm.cell_dofs(3, (2, 2, 2), 2, 1, 8)  # cell 8 of 8
    with _pytest.raises(fcm.FcmError):
        fcm.cell_dofs(4, (2, 2, 2), 2, 1, 0)


def _oracle_topology(prob):
    from oracle.mlhp import MlhpSpace, mesh_for, schwarz_blocks
    import numpy as np
    space = MlhpSpace(mesh_for(prob), prob["p"], 1)
    d = prob["dim"]
    level, t, q = [], [], []
    for k, tt, qs in space.funcs:
        level.append(k)
        t.append(list(tt) + [0] * (3 - d))
        qq, i = [0, 0, 0], 0
        for a in range(d):
            if tt[a] % 2:
                qq[a] = qs[i]
                i += 1
        q.append(qq)
    leaves, lf = [], []
    for k, e in space.mesh.leaves():
        leaves.append((k, list(e) + [0] * (3 - d)))
        lf.append(np.concatenate([ids for _, _, _, ids in space.leaf_functions(k, e)]).tolist())
    patches = [b.tolist() for b in schwarz_blocks(space, np.arange(space.M), "patchwise")]
    return level, t, q, leaves, lf, patches


@pytest.mark.parametrize("make", [
    lambda fi: dict(fi.poisson2d_circle(cells=8, p=2), overlay_levels=3),
    lambda fi: dict(fi.poisson2d_circle(cells=6, p=1), overlay_levels=3),
    lambda fi: dict(fi.elasticity3d_voids(cells=4, p=1, n_voids=3), overlay_levels=1),
    lambda fi: dict(fi.poisson2d_circle(cells=5, p=3, radius=0.3), overlay_levels=2),
    lambda fi: fi.perforated_plate(cells=8, p=2, overlay_levels=2),
    lambda fi: dict(fi.poisson3d_sphere(cells=4, p=2, radius=0.3), overlay_levels=2),
    lambda fi: dict(fi.batch_instance(3), cells=(3, 3, 3), p=2, overlay_levels=1),
])
def test_overlay_topology_matches_the_oracle(make):
    """fcm_mlhp_* (host functions, no GPU): refinement, active functions and
    their numbering, the per-leaf function lists and the patches, bit-exact
    against oracle/mlhp.py."""
    import fcm_inputs as fi
    from paper_2010_00881_gb300 import fcm
    prob = make(fi)
    ov = fcm.Overlay(prob)
    level, t, q, leaves, lf, patches = _oracle_topology(prob)
    assert ov.n_functions == len(level) and ov.n_leaves == len(leaves)
    assert ov.level.tolist() == level
    assert ov.t.tolist() == t and ov.q.tolist() == q
    assert [(int(k), e.tolist()) for k, e in zip(ov.leaf_level, ov.leaf_index)] == leaves
    off = ov.leaf_offsets
    assert [ov.leaf_functions[off[i]:off[i + 1]].tolist() for i in range(len(leaves))] == lf
    po = ov.patch_offsets
    assert [ov.patch_functions[po[i]:po[i + 1]].tolist() for i in range(len(po) - 1)] == patches
    assert max(ov.leaf_level) == prob["overlay_levels"]


def test_overlay_topology_rejects_invalid_input():
    import fcm_inputs as fi
    from paper_2010_00881_gb300 import fcm
    base = dict(fi.poisson2d_circle(cells=8, p=2), overlay_levels=2)
    for bad in (dict(base, overlay_levels=11), dict(base, p=0), dict(base, p=9),
                dict(base, cells=(1 << 18, 2), overlay_levels=2),
                dict(base, geometry=dict(kind="ellipsoid", center=(0.5, 0.5, 0.5),
                                         axes=(0.3, 0.3, 0.3),
                                         rot=[[1, 0, 0], [0, 1, 0], [0, 0, 1]])),
                dict(base, geometry=dict(kind="ball", center=(0.5, float("nan")), radius=0.3)),
                dict(base, hi=(1.0, float("inf")))):
        with pytest.raises(fcm.FcmError) as e:
            fcm.Overlay(bad)
        assert e.value.status == fcm.FCM_E_INVALID


def test_restriction_1d_matches_interpolation():
    """fcm_mlhp_restriction_1d against the oracle's basis: the ancestor's
    modes at the sub-interval's Gauss points, solved in the sub-interval's
    own modes."""
    import numpy as np
    from oracle.basis import basis_1d, gauss_legendre
    from paper_2010_00881_gb300 import fcm
    for p in range(1, 7):
        xi, _ = gauss_legendre(p + 1)
        V = basis_1d(p, xi)[0].T
        for dk in range(4):
            s = 2.0 ** -dk
            for pos in range(1 << dk):
                c = -1.0 + s * (2 * pos + 1)
                ref = np.linalg.solve(V, basis_1d(p, c + s * xi)[0].T)
                S = fcm.restriction_1d(p, dk, pos)
                assert np.abs(S - ref).max() <= 1e-12, (p, dk, pos)
        assert np.array_equal(fcm.restriction_1d(p, 0, 0), np.eye(p + 1))
    for bad in ((0, 0, 0), (9, 0, 0), (2, -1, 0), (2, 2, 4), (2, 11, 0)):
        with pytest.raises(fcm.FcmError):
            fcm.restriction_1d(*bad)


@pytest.mark.parametrize("make", [
    lambda fi: dict(fi.poisson2d_circle(cells=6, p=3, radius=0.3), overlay_levels=3),
    lambda fi: fi.poisson3d_sphere_mlhp(cells=3, p=2, overlay_levels=2),
])
def test_leaf_transform_is_a_kronecker_product_of_restrictions(make):
    """On every leaf, the leaf's own modal coefficients of its functions (the
    oracle, by interpolation) are the Kronecker products of the per-axis
    restrictions of their ancestors, columns in the leaf's function order."""
    import numpy as np
    import fcm_inputs as fi
    from oracle.assembly import shape_functions
    from oracle.mlhp import MlhpSpace, mesh_for
    from oracle.quadrature import leaf_rule
    from paper_2010_00881_gb300 import fcm
    prob = make(fi)
    space = MlhpSpace(mesh_for(prob), prob["p"], 1)
    p, d = space.p, prob["dim"]
    R = {(dk, pos): fcm.restriction_1d(p, dk, pos) for dk in range(4) for pos in range(1 << dk)}
    modes = space.modes
    for k, e in space.mesh.leaves():
        x0, x1 = space.mesh.box(k, e)
        pts, _ = leaf_rule(x0, x1, p)
        V, _ = shape_functions(p, x0, x1, pts)
        ids, N, _ = space.eval_on_leaf(k, e, pts)
        T = np.linalg.solve(V, N)
        cols = []
        for j, _, mcols, _ in space.leaf_functions(k, e):
            dk = k - j
            S = [R[(dk, e[a] % (1 << dk))] for a in range(d)]
            for m in mcols:
                js = modes[m]
                col = np.ones(1)
                for a in reversed(range(d)):      # x fastest: kron(z, y, x)
                    col = np.kron(col, S[a][:, js[a]])
                cols.append(col)
        assert np.abs(np.column_stack(cols) - T).max() <= 1e-12


@pytest.mark.parametrize("make", [
    lambda fi: dict(fi.poisson2d_circle(cells=8, p=3), overlay_levels=3),
    lambda fi: dict(fi.poisson2d_circle(cells=8, p=1), overlay_levels=2),
    lambda fi: fi.perforated_plate(cells=8, p=2, overlay_levels=3),
    lambda fi: fi.poisson3d_sphere_mlhp(cells=4, p=2, overlay_levels=2),
    lambda fi: dict(fi.poisson2d_circle(cells=4, p=2), overlay_levels=0),
    # a hole instead of an inclusion: the same leaves, inside and outside swapped
    lambda fi: dict(fi.poisson2d_circle(cells=8, p=2), overlay_levels=2,
                    geometry=dict(kind="ball", center=(0.5, 0.5), radius=0.4, complement=True)),
])
def test_overlay_leaf_classes_and_levels_match_the_oracle(make):
    import numpy as np
    import fcm_inputs as fi
    from oracle.geometry import classify_box
    from oracle.mlhp import MlhpSpace, hp_level_sets, mesh_for
    from paper_2010_00881_gb300 import fcm
    prob = make(fi)
    ov = fcm.Overlay(prob)
    space = MlhpSpace(mesh_for(prob), prob["p"], 1)
    cls = [classify_box(prob["geometry"], *space.mesh.box(k, e)) for k, e in space.mesh.leaves()]
    assert ov.leaf_classes.tolist() == cls
    sets = hp_level_sets(space)
    n = len(sets)
    assert ov.n_levels == n
    for i, s in enumerate(sets):
        assert np.flatnonzero(ov.coarsest <= n - 1 - i).tolist() == s.tolist(), i


def test_descriptors_refuse_what_the_library_lacks():
    """Problem features without a library descriptor raise instead of being
    dropped silently (spaces other than tensor and trunk, removal of fully
    fictitious cells without trunk elements); overlays, patchwise blocks and
    trunk elements with the Jacobi smoother reach the library (which rejects
    them in fcm_setup)."""
    import fcm_inputs as fi
    from paper_2010_00881_gb300 import fcm
    base = fi.poisson3d_sphere(cells=4, p=2)
    for bad in (dict(base, space="serendipity"), dict(base, drop_outside=True),
                fi.popcorn(cells=4, space="tensor"), dict(base, smoother="gauss_seidel")):
        with pytest.raises(ValueError):
            fcm.descriptors(bad)
    g, _, _, _, _ = fcm.descriptors(fi.popcorn(cells=4))
    assert g.space == fcm.SPACE_TRUNK and g.drop_outside == 1
    g, _, _, op, _ = fcm.descriptors(fi.poisson3d_sphere_mlhp(cells=4))
    assert g.overlay_levels == 3 and op.smoother == 1
    g, _, _, op, _ = fcm.descriptors(dict(base, space="trunk", smoother="jacobi"))
    assert g.space == fcm.SPACE_TRUNK and op.smoother == 2
    g, _, _, _, _ = fcm.descriptors(fi.popcorn(cells=4, space="tensor", drop_outside=False))
    assert g.space == fcm.SPACE_TENSOR
    g, _, _, _, _ = fcm.descriptors(fi.popcorn(cells=4, drop_outside=False))
    assert g.space == fcm.SPACE_TRUNK
    _, gm, _, _, _ = fcm.descriptors(base)
    assert gm.complement == 0
    _, gm, _, _, _ = fcm.descriptors(dict(base, geometry=dict(base["geometry"], complement=True)))
    assert gm.complement == 1


def test_quadrature_descriptor():
    """The leaf-sum scheme of the cell integration reaches fcm_physics:
    point sums by default, sum factorisation on request, anything else
    refused before the library is called."""
    import fcm_inputs as fi
    from paper_2010_00881_gb300 import fcm
    base = fi.poisson3d_sphere(cells=4, p=3)
    _, _, ph, _, _ = fcm.descriptors(base)
    assert ph.quadrature == fcm.QUAD_POINTS == 0
    _, _, ph, _, _ = fcm.descriptors(dict(base, quadrature="sumfact"))
    assert ph.quadrature == fcm.QUAD_SUMFACT == 1
    with pytest.raises(ValueError):
        fcm.descriptors(dict(base, quadrature="gauss"))
