"""Parity at full size, in the launch configuration the throughput runs use.

The oracle cannot assemble these problems whole, so sampled rows of the
operator are checked: y_I = sum over the cells c that hold DOF I of
K_c[l_c(I), :] x[dofs(c)], with K_c the oracle's element matrix (weak form,
Sec. 2; space-tree quadrature of cut cells, Sec. 2.2).  Samples cover
interior bubble DOFs (one cell) of cut, inside and outside cells, and
vertex DOFs of cut cells (up to 2^d cells, stored and shared matrices
mixed).  Bars, per sampled row, relative to s_I = sum_c |K_c[l, :]| |x|:
FP64 1e-11 (two quadrature summation orders), mixed 1e-5 (FP32 data, shared
matrices on the tensor cores in 3xTF32).

The solves are checked by properties that hold at any size: the true
relative residual (FP64 operator, itself checked above) below the
tolerance, and the mixed solve taking the FP64 solve's iteration count +-1.
"""
import numpy as np
import pytest

import fcm_inputs as fi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from oracle.assembly import element_system, nfields  # noqa: E402
from oracle.geometry import CUT, INSIDE, OUTSIDE  # noqa: E402
from oracle.grid import cell_dofs  # noqa: E402
from paper_2010_00881_gb300 import FCM_FP64, FCM_MIXED, Solver  # noqa: E402

WORKLOADS = {
    # the throughput workload: 32^3 cells, p = 3, sphere, 912,673 DOFs
    "sphere32_p3": lambda: fi.poisson3d_sphere(),
    # 64^3 cells, p = 2, block with 64 spherical voids, 6.4M DOFs
    "elastic64_p2": lambda: fi.elasticity3d_voids(p=2),
    # the popcorn of Sec. 4.3.2 on the paper's coarsest grid, 96^3 cells of
    # (-1, 1)^3, p = 3, tensor-product space on all cells: 24.1M DOFs
    "popcorn96_p3": lambda: fi.popcorn(cells=96, p=3, space="tensor", drop_outside=False),
}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def big(request):
    prob = WORKLOADS[request.param]()
    s = Solver(prob)
    yield request.param, prob, s
    s.close()


def _cells_of(cls, kind, count, rng, C):
    idx = np.flatnonzero(cls == kind)
    pick = rng.choice(idx, size=min(count, len(idx)), replace=False)
    out = []
    for c in pick:
        cx = int(c % C[0])
        cy = int((c // C[0]) % C[1])
        cz = int(c // (C[0] * C[1]))
        out.append((cx, cy, cz)[: len(C)])
    return out


def _samples(prob, cls, rng):
    """(DOF, [(cell, local index)]) for the sampled rows."""
    d, C, p = prob["dim"], prob["cells"], prob["p"]
    nf = nfields(prob)
    P1 = p + 1
    nls = P1 ** d
    bubble = sum(2 * P1 ** a for a in range(d))  # local modes (2, 2, ...)
    out = []
    for kind, count in ((CUT, 6), (INSIDE, 3), (OUTSIDE, 2)):
        for cell in _cells_of(cls, kind, count, rng, C):
            f = int(rng.integers(nf))
            l = f * nls + bubble
            out.append((int(cell_dofs(d, C, p, cell, nf)[l]), [(cell, l)]))
    for cell in _cells_of(cls, CUT, 3, rng, C):
        I = int(cell_dofs(d, C, p, cell, nf)[0])  # vertex (0, 0, ...) of field 0
        holders = []
        for off in np.ndindex(*([2] * d)):
            nb = tuple(cell[a] - off[a] for a in range(d))
            if min(nb) < 0:
                continue
            dofs = cell_dofs(d, C, p, nb, nf)
            hit = np.flatnonzero(dofs == I)
            if len(hit):
                holders.append((nb, int(hit[0])))
        out.append((I, holders))
    return out


def test_sampled_operator_rows(big):
    name, prob, s = big
    rng = np.random.default_rng(7)
    cls = s.cell_classes()
    d, C, p = prob["dim"], prob["cells"], prob["p"]
    nf = nfields(prob)
    x = fi.random_vector(s.ndofs, seed=3)
    xt = torch.from_numpy(x).cuda()
    y64 = s.apply(xt).cpu().numpy()
    y32 = s.apply(xt, prec=FCM_MIXED).cpu().numpy()
    cache = {}
    for I, holders in _samples(prob, cls, rng):
        ref = 0.0
        scale = 0.0
        for cell, l in holders:
            if cell not in cache:
                cache[cell] = element_system(prob, cell)[0]
            K = cache[cell]
            xd = x[cell_dofs(d, C, p, cell, nf)]
            ref += K[l] @ xd
            scale += np.abs(K[l]) @ np.abs(xd)
        assert abs(y64[I] - ref) <= 1e-11 * scale, (name, I, y64[I], ref, scale)
        assert abs(y32[I] - ref) <= 1e-5 * scale, (name, I, y32[I], ref, scale)


def test_solves(big):
    name, prob, s = big
    _, i64 = s.pcg(rtol=1e-8, prec=FCM_FP64)
    _, i32 = s.pcg(rtol=1e-8, prec=FCM_MIXED)
    assert i64["relres_true"] <= 1e-8 and i32["relres_true"] <= 1e-8
    assert abs(i32["iters"] - i64["iters"]) <= 1, (i32["iters"], i64["iters"])
