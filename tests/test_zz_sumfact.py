"""Sum-factorised leaf sums (fcm_physics.quadrature = FCM_QUAD_SUMFACT)
against the point sums on the device: the same Gauss points and weights, so
the load (summed point by point in both) is bit for bit the same and A x
agrees to rounding (1e-13 relative); Poisson p = 2, 3, 4, 8 and elasticity
p = 2, 3 in 2D and 3D, and the operator of an overlay mesh."""
import numpy as np
import pytest

import fcm_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2010_00881_gb300 import FCM_FP64, Solver  # noqa: E402
from paper_2010_00881_gb300 import fcm as F  # noqa: E402

CASES = {
    "circle8_p2": lambda: fi.poisson2d_circle(cells=8, p=2),
    "circle4_p8": lambda: fi.poisson2d_circle(cells=4, p=8),
    "sphere4_p3": lambda: fi.poisson3d_sphere(cells=4, p=3),
    "sphere3_p4": lambda: fi.poisson3d_sphere(cells=3, p=4),
    "plate8_p3": lambda: fi.perforated_plate(cells=8, p=3, overlay_levels=0),
    "voids4_p2": lambda: fi.elasticity3d_voids(cells=4, p=2, n_voids=3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_sumfact_equals_point_sums(name):
    prob = CASES[name]()
    a = Solver(prob)
    b = Solver(dict(prob, quadrature="sumfact"))
    try:
        ra, rb = a.rhs().cpu().numpy(), b.rhs().cpu().numpy()
        assert np.array_equal(ra, rb), name
        x = torch.from_numpy(fi.random_vector(a.ndofs, seed=1)).cuda()
        ya = a.apply(x, prec=FCM_FP64).cpu().numpy()
        yb = b.apply(x, prec=FCM_FP64).cpu().numpy()
        err = np.linalg.norm(ya - yb) / np.linalg.norm(ya)
        print(f"{name}: {err:.2e}")
        assert err <= 1e-13, (name, err)
    finally:
        a.close()
        b.close()


def test_sumfact_overlay_operator():
    prob = fi.poisson3d_sphere_mlhp(cells=4, p=2, overlay_levels=2)
    a, b = F.MlhpOperator(prob), F.MlhpOperator(dict(prob, quadrature="sumfact"))
    try:
        x = torch.from_numpy(fi.random_vector(a.ndofs, seed=1)).cuda()
        ya, yb = a.apply(x).cpu().numpy(), b.apply(x).cpu().numpy()
        assert np.linalg.norm(ya - yb) <= 1e-13 * np.linalg.norm(ya)
    finally:
        a.close()
        b.close()
