"""The multi-level hp operator on the GPU (refinement by superposition,
Sec. 2.2) through the C ABI, against the oracle's leaf assembly
(oracle.mlhp.assemble_mlhp).

The device integrates every leaf's box with the cell kernels and maps it to
the leaf's functions by the Kronecker product of 1D restrictions
(K_L = T^T K_box T); the oracle integrates the functions of every ancestor
on the leaf directly.  The two are the same quadrature of the same
polynomials, so the load and A x agree to rounding: 1e-12 relative, the
FP64 bar.  Cases: 2D Poisson with three overlays on a cut circle, the 3D
sphere with two overlays (p = 2), the elastic perforated plate (box-face
Dirichlet and traction terms on refined leaves), a 3D elastic block with
voids and one overlay, and a hole (complement domain) with two overlays.

Without overlays the same path is the patchwise additive Schwarz smoother
on uniform grids, checked against the uniform oracle hierarchy as well.
"""
import numpy as np
import pytest

import fcm_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from oracle.mlhp import assemble_mlhp  # noqa: E402
from paper_2010_00881_gb300 import fcm as F  # noqa: E402

CASES = {
    "circle8_p2_k3": lambda: dict(fi.poisson2d_circle(cells=8, p=2), overlay_levels=3),
    "sphere4_p2_k2": lambda: fi.poisson3d_sphere_mlhp(cells=4, p=2, overlay_levels=2),
    "plate8_p2_k2": lambda: fi.perforated_plate(cells=8, p=2, overlay_levels=2),
    "voids4_p1_k1": lambda: dict(fi.elasticity3d_voids(cells=4, p=1, n_voids=3), overlay_levels=1),
    "hole8_p3_k2": lambda: dict(fi.poisson2d_circle(cells=8, p=3), overlay_levels=2,
                                geometry=dict(kind="ball", center=(0.5, 0.5), radius=0.4,
                                              complement=True)),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    prob = CASES[request.param]()
    A, b, space = assemble_mlhp(prob)
    op = F.MlhpOperator(prob)
    yield request.param, prob, A, b, space, op
    op.close()


def test_sizes(case):
    name, prob, A, b, space, op = case
    assert op.ndofs == A.shape[0] == space.N


def test_load(case):
    name, prob, A, b, space, op = case
    bg = op.rhs().cpu().numpy()
    assert np.abs(bg - b).max() <= 1e-12 * np.abs(b).max(), name


def test_apply(case):
    name, prob, A, b, space, op = case
    x = fi.random_vector(op.ndofs, seed=3)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = A @ x
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref), name
    # bit for bit reproducible
    y2 = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y, y2)


def test_apply_is_symmetric(case):
    name, prob, A, b, space, op = case
    u = fi.random_vector(op.ndofs, seed=4)
    v = fi.random_vector(op.ndofs, seed=5)
    Au = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    Av = op.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert abs(v @ Au - u @ Av) <= 1e-12 * (np.abs(v) @ np.abs(Au) + 1e-300)


# ---------------------------------------------------------------------------
# The hp-multigrid of overlay meshes (Sec. 3.2, Fig. hpmultigrid; the Q1
# h-levels of the Remark of Sec. 3.2 below the base grid) against
# oracle.mlhp.MlhpHierarchy: level sizes exact, omega 1e-6, the V-cycle
# within 1e-12 + 50 x the LU-inverse noise floor (energy norm), PCG
# iteration counts +-1 and the oracle's true residual.

from oracle import multigrid as mg  # noqa: E402
from oracle.mlhp import MlhpHierarchy  # noqa: E402
from parity_helpers import Noise  # noqa: E402

SOLVER_CASES = {
    # hierarchies ending at the base grid (base cells <= coarse_cells)
    "circle4_p2_k3_patch": lambda: dict(fi.poisson2d_circle(cells=4, p=2), overlay_levels=3,
                                        smoother="patchwise"),
    "circle4_p3_k2_elem": lambda: dict(fi.poisson2d_circle(cells=4, p=3), overlay_levels=2,
                                       smoother="elementwise"),
    "sphere4_p1_k2_patch": lambda: fi.poisson3d_sphere_mlhp(cells=4, p=1, overlay_levels=2),
    # Q1 h-levels below the base grid (Galerkin, ragged halving 10 -> 5 -> 3)
    "circle8_p2_k2_patch": lambda: dict(fi.poisson2d_circle(cells=8, p=2), overlay_levels=2,
                                        smoother="patchwise"),
    "circle10_p2_k1_elem": lambda: dict(fi.poisson2d_circle(cells=10, p=2), overlay_levels=1,
                                        smoother="elementwise"),
    "plate8_p2_k2_patch": lambda: dict(fi.perforated_plate(cells=8, p=2, overlay_levels=2),
                                       smoother="patchwise"),
    "sphere6_p1_k1_patch": lambda: fi.poisson3d_sphere_mlhp(cells=6, p=1, overlay_levels=1),
    # no overlays: patchwise blocks on uniform grids (12 -> 6 -> 3 Q1 levels)
    "circle8_p3_k0_patch": lambda: dict(fi.poisson2d_circle(cells=8, p=3), overlay_levels=0,
                                        smoother="patchwise"),
    "circle12_p2_k0_patch": lambda: dict(fi.poisson2d_circle(cells=12, p=2), overlay_levels=0,
                                         smoother="patchwise"),
    "sphere4_p2_k0_patch": lambda: dict(fi.poisson3d_sphere(cells=4, p=2, radius=0.3),
                                        overlay_levels=0, smoother="patchwise"),
}
UNIFORM_CASES = [k for k in SOLVER_CASES if "_k0_" in k]


@pytest.fixture(scope="module", params=list(SOLVER_CASES))
def solver_case(request):
    prob = SOLVER_CASES[request.param]()
    H = MlhpHierarchy(prob)
    op = F.MlhpOperator(prob)
    op.prepare()
    yield request.param, prob, H, op
    op.close()


def _rel_a(A, a, b):
    e = a - b
    return np.sqrt(max(e @ (A @ e), 0.0)) / np.sqrt(b @ (A @ b))


def test_hierarchy_levels(solver_case):
    name, prob, H, op = solver_case
    assert len(op.levels) == len(H.levels)
    for l, (info, lv) in enumerate(zip(op.levels, H.levels)):
        assert info["ndofs"] == lv.N, (name, l)
        if l > 0:
            assert abs(info["omega"] - lv.omega) <= 1e-6 * lv.omega, (name, l, info, lv.omega)
            assert info["n_blocks"] == sum(len(IDX) for IDX, _ in lv.groups), (name, l)


def test_vcycle(solver_case):
    name, prob, H, op = solver_case
    r = fi.random_vector(op.ndofs, seed=2)
    z = op.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    zr = H.vcycle(r)
    bar = 1e-12 + 50.0 * _rel_a(H.A, Noise(H).vcycle(r), zr)
    err = _rel_a(H.A, z, zr)
    print(f"overlay V-cycle {name}: {err:.2e} (bar {bar:.2e})")
    assert err <= bar, (name, err, bar)


def test_pcg(solver_case):
    name, prob, H, op = solver_case
    _, ko, _ = mg.pcg(H.A, H.b, H.vcycle, rtol=1e-8)
    x, info = op.pcg(rtol=1e-8)
    x = x.cpu().numpy()
    assert info["relres_true"] <= 1e-8
    assert np.linalg.norm(H.b - H.A @ x) / np.linalg.norm(H.b) <= 1.01e-8
    assert abs(info["iters"] - ko) <= 1, (name, info["iters"], ko)


@pytest.mark.parametrize("name", UNIFORM_CASES)
def test_uniform_grid_patchwise_equals_uniform_hierarchy(name):
    """Without overlays the device's hp-multigrid is the uniform-grid
    hierarchy of Sec. 3.1 with the patchwise blocks of Sec. 3.3.1: its
    V-cycle equals the uniform oracle's (oracle.multigrid.Hierarchy, grid
    numbering, the omega per level taken from the device, whose power-method
    start vector follows the overlay numbering) within 1e-12 + 50 x the
    LU-inverse noise floor, and PCG takes the uniform oracle's iteration
    count +-1."""
    from oracle.mlhp import MlhpSpace, mesh_for
    from oracle.multigrid import Hierarchy
    from parity_helpers import uniform_index
    prob = SOLVER_CASES[name]()
    U = Hierarchy(prob)
    op = F.MlhpOperator(prob)
    try:
        op.prepare()
        assert [info["ndofs"] for info in op.levels] == [lv.N for lv in U.levels]
        for info, lv in zip(op.levels[1:], U.levels[1:]):
            assert abs(info["omega"] - lv.omega) <= 0.03 * lv.omega
            lv.omega = info["omega"]
        perm = uniform_index(MlhpSpace(mesh_for(prob), prob["p"], 1))
        r = fi.random_vector(op.ndofs, seed=2)
        ru = np.zeros_like(r)
        ru[perm] = r
        z = np.zeros_like(r)
        z[perm] = op.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
        zu = U.vcycle(ru)
        bar = 1e-12 + 50.0 * _rel_a(U.A, Noise(U).vcycle(ru), zu)
        err = _rel_a(U.A, z, zu)
        print(f"uniform patchwise V-cycle {name}: {err:.2e} (bar {bar:.2e})")
        assert err <= bar, (name, err, bar)
        _, ku, _ = mg.pcg(U.A, U.b, U.vcycle, rtol=1e-8)
        x, info = op.pcg(rtol=1e-8)
        assert abs(info["iters"] - ku) <= 1, (name, info["iters"], ku)
        xu = np.zeros_like(r)
        xu[perm] = x.cpu().numpy()
        assert np.linalg.norm(U.b - U.A @ xu) / np.linalg.norm(U.b) <= 1.01e-8
    finally:
        op.close()
