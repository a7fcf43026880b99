"""Trunk-space elements (Sec. 4.3) on the GPU, with and without removal of
the fully fictitious cells (Sec. 4.3.2), through the C ABI, against the
oracle's trunk hierarchy (oracle.trunk.TrunkHierarchy).

The library keeps the tensor layout and removes the non-trunk modes from the
system; the oracle numbers the trunk DOFs consecutively.  A library vector
maps to the oracle's by the kept tensor indices (fields stacked), and every
library output is zero on the removed modes.  Bars as for the tensor space:
counts exact, load and FP64 apply <= 1e-12, FP32 apply <= 1e-5, V-cycle
within 1e-12 + 50 x the LU-inverse noise floor (energy norm), the mixed
V-cycle within 10 x its error measured on a GB300, PCG iterations
+-1 in both precisions, parity-mode solutions (rtol 1e-11) within 1e-8
relative L2 over the physical domain.
"""
import numpy as np
import pytest

import fcm_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from oracle import multigrid as mg  # noqa: E402
from oracle.grid import m_1d  # noqa: E402
from oracle.trunk import TrunkHierarchy, trunk_global_mask  # noqa: E402
from paper_2010_00881_gb300 import FCM_FP64, FCM_MIXED, Solver  # noqa: E402
from paper_2010_00881_gb300 import fcm as F  # noqa: E402
from parity_helpers import Noise, PhysField  # noqa: E402


def _trunk(prob):
    return dict(prob, space="trunk")


def _drop(prob):
    return dict(prob, space="trunk", drop_outside=True)


CASES = {
    "sphere4_p3": lambda: _trunk(fi.poisson3d_sphere(cells=4, p=3)),
    "sphere5_p2": lambda: _trunk(fi.poisson3d_sphere(cells=5, p=2)),
    "circle8_p4": lambda: _trunk(fi.poisson2d_circle(cells=8, p=4)),
    "elastic4_p2": lambda: _trunk(fi.elasticity3d_voids(cells=4, p=2, n_voids=3, seed=1)),
    # fully fictitious cells removed as well (the paper's popcorn setting)
    "sphere6_p3_drop": lambda: _drop(fi.poisson3d_sphere(cells=6, p=3)),
    "circle9_p4_drop": lambda: _drop(fi.poisson2d_circle(cells=9, p=4)),
    "popcorn8_p2_drop": lambda: fi.popcorn(cells=8, p=2),
}


# Energy-norm error of the mixed V-cycle against the oracle's FP64 V-cycle
# (random residual, seed 2) measured on a GB300; the test bar is 10 x these.
MIXED_VCYCLE = {"sphere4_p3": 5.5e-7, "sphere5_p2": 1.1e-6, "circle8_p4": 3.7e-5,
                "elastic4_p2": 3.7e-7, "sphere6_p3_drop": 2.0e-5, "circle9_p4_drop": 2.8e-5,
                "popcorn8_p2_drop": 1.6e-6}


def _level_index(prob, nf, pc, kept):
    """Library indices (tensor layout of degree pc, fields stacked) of the
    oracle's DOFs of the trunk p-level of degree pc, in the oracle's order;
    kept: the finest level's kept scalar ids (degree-p layout)."""
    d, C, p = prob["dim"], prob["cells"], prob["p"]
    ts = kept[trunk_global_mask(d, C, p, pc)[kept]]          # ids in the degree-p layout
    out = np.zeros(len(ts), dtype=np.int64)
    rem = ts.copy()
    stride = 1
    for a in range(d):
        ia = rem % m_1d(C[a], p)
        rem //= m_1d(C[a], p)
        out += ia * stride
        stride *= m_1d(C[a], pc)
    Mpc = stride
    return np.concatenate([f * Mpc + out for f in range(nf)]), nf * Mpc


class Case:
    def __init__(self, name):
        self.name = name
        self.prob = CASES[name]()
        self.H = TrunkHierarchy(self.prob)
        self.s = Solver(self.prob)
        self.nf = self.H.space.nf
        self.kept = self.H.space.tensor_index
        self.idx, self.N = _level_index(self.prob, self.nf, self.prob["p"], self.kept)

    def to_lib(self, xo, idx=None, N=None):
        idx = self.idx if idx is None else idx
        x = np.zeros(self.N if N is None else N)
        x[idx] = xo
        return x

    def run(self, fn, x):
        return fn(torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    c = Case(request.param)
    yield c
    c.s.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _rel_a(A, a, b):
    e = a - b
    return np.sqrt(max(e @ (A @ e), 0.0)) / np.sqrt(b @ (A @ b))


def _removed(c, y, idx=None):
    keep = np.zeros(len(y), dtype=bool)
    keep[c.idx if idx is None else idx] = True
    return np.abs(y[~keep]).max(initial=0.0)


def test_levels_and_dofs(case):
    c = case
    s, H = c.s, c.H
    assert s.num_levels() == len(H.levels)
    for l, lv in enumerate(H.levels):
        info = s.level_info(l)
        assert info["ndofs_active"] == lv.N, (c.name, l, info["ndofs_active"], lv.N)
        assert info["p"] == lv.p
        if info["p"] == 1 and not c.prob.get("drop_outside"):
            assert info["ndofs"] == lv.N
        if l > 0:
            assert abs(info["omega"] - lv.omega) <= 1e-6 * lv.omega, (l, info["omega"], lv.omega)
        assert info["kron_operator"] == 0


def test_rhs(case):
    c = case
    b = c.s.rhs().cpu().numpy()
    assert _removed(c, b) == 0.0
    assert np.abs(b[c.idx] - c.H.b).max() <= 1e-12 * np.abs(c.H.b).max()


def test_apply(case):
    c = case
    x = fi.random_vector(c.N, seed=1)    # removed modes too: ignored
    ref = c.H.A @ x[c.idx]
    y = c.run(c.s.apply, x)
    assert _removed(c, y) == 0.0
    assert _rel(y[c.idx], ref) <= 1e-12
    y32 = c.run(lambda t: c.s.apply(t, prec=FCM_MIXED), x)
    assert _removed(c, y32) == 0.0
    assert _rel(y32[c.idx], ref) <= 1e-5, _rel(y32[c.idx], ref)


def test_level_operators(case):
    c = case
    s, H = c.s, c.H
    noise = Noise(H)
    for l, lv in enumerate(H.levels):
        info = s.level_info(l)
        if info["is_h_level"] or l == 0:
            continue
        idx, N = _level_index(c.prob, c.nf, lv.p, c.kept)
        xo = fi.random_vector(lv.N, seed=10 + l)
        x = c.to_lib(xo, idx, N)
        y = s.level_op(l, F.OP_APPLY, torch.from_numpy(x).cuda(), N).cpu().numpy()
        assert _removed(c, y, idx) == 0.0
        assert _rel(y[idx], lv.A @ xo) <= 1e-12, ("A", l)
        z = s.level_op(l, F.OP_SMOOTHER, torch.from_numpy(x).cuda(), N).cpu().numpy()
        assert _removed(c, z, idx) == 0.0
        zr = lv.smoother(xo)
        bar = 1e-12 + 50.0 * _rel_a(lv.A, noise.smoother(l, xo), zr)
        assert _rel_a(lv.A, z[idx], zr) <= bar, ("M", l, _rel_a(lv.A, z[idx], zr), bar)


def test_vcycle(case):
    c = case
    H = c.H
    ro = fi.random_vector(H.A.shape[0], seed=2)
    zr = H.vcycle(ro)
    z = c.run(c.s.vcycle, c.to_lib(ro))
    assert _removed(c, z) == 0.0
    bar = 1e-12 + 50.0 * _rel_a(H.A, Noise(H).vcycle(ro), zr)
    assert _rel_a(H.A, z[c.idx], zr) <= bar, (_rel_a(H.A, z[c.idx], zr), bar)
    z32 = c.run(lambda t: c.s.vcycle(t, prec=FCM_MIXED), c.to_lib(ro))
    assert _removed(c, z32) == 0.0
    err = _rel_a(H.A, z32[c.idx], zr)
    print(f"trunk mixed V-cycle {c.name}: {err:.2e}")
    assert err <= 10.0 * MIXED_VCYCLE[c.name], (c.name, err)


def test_pcg_iterations(case):
    c = case
    H = c.H
    _, ko, _ = mg.pcg(H.A, H.b, H.vcycle, rtol=1e-8)
    for prec in (FCM_FP64, FCM_MIXED):
        x, info = c.s.pcg(rtol=1e-8, prec=prec)
        x = x.cpu().numpy()
        assert info["relres_true"] <= 1e-8
        assert _removed(c, x) == 0.0
        assert np.linalg.norm(H.b - H.A @ x[c.idx]) / np.linalg.norm(H.b) <= 1.01e-8
        assert abs(info["iters"] - ko) <= 1, (c.name, prec, info["iters"], ko)


def test_solution_parity_mode(case):
    c = case
    H = c.H
    xo, _, _ = mg.pcg(H.A, H.b, H.vcycle, rtol=1e-11)
    pf = PhysField(dict(c.prob, space="tensor"))
    xo_lib = c.to_lib(xo)
    for prec in (FCM_FP64, FCM_MIXED):
        x, _ = c.s.pcg(rtol=1e-11, maxit=500, prec=prec)
        x = x.cpu().numpy()
        e = pf.rel(x, xo_lib)
        print(f"trunk parity mode {c.name} prec {prec}: phys {e:.2e}")
        assert e <= 1e-8, (c.name, prec, e)


def test_user_rhs_ignores_removed_modes(case):
    """A caller's b with values on the removed modes solves the system of
    its trunk entries: the assembled load plus noise there gives the solve
    of the assembled load, bit for bit."""
    c = case
    b = c.s.rhs().cpu().numpy()
    keep = np.zeros(c.N, dtype=bool)
    keep[c.idx] = True
    b[~keep] = fi.random_vector(int((~keep).sum()), seed=6)
    x0, i0 = c.s.pcg(rtol=1e-8)
    x1, i1 = c.s.pcg(b=torch.from_numpy(b).cuda(), rtol=1e-8)
    assert i1["iters"] == i0["iters"]
    assert torch.equal(x0, x1)
    assert _removed(c, x1.cpu().numpy()) == 0.0
