"""Pins of the oracle's element matrices and global assembly (Eq. weakform).

* An uncut cell's stiffness equals the Kronecker sum of the exact 1D
  matrices (closed form from test_oracle_basis), for any cell shape.
* Elasticity element matrices annihilate exactly the rigid-body modes.
* The nodal modes form a partition of unity, so the nodal load entries sum
  to the alpha-weighted volume integral of f.
* The assembled matrix is symmetric positive definite.
* Manufactured solutions converge at the expected rates under h- and
  p-refinement (body-fitted square, exact quadrature).
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import fcm_inputs as fi
from oracle.assembly import (assemble, element_system, elasticity_C, exact_solution,
                             shape_functions)
from oracle.basis import element_1d_matrices
from oracle.geometry import INSIDE, OUTSIDE
from oracle.grid import all_cells, cell_box, cell_dofs, m_1d
from oracle.quadrature import leaf_rule


def kron_sum(mats_K, mats_M):
    """sum_a (x)_b (K if a == b else M), x fastest (rightmost factor)."""
    d = len(mats_K)
    out = 0
    for a in range(d):
        term = np.ones((1, 1))
        for b in reversed(range(d)):
            term = np.kron(term, mats_K[b] if a == b else mats_M[b])
        out = out + term
    return out


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 1), (3, 3)])
def test_uncut_cell_is_kronecker_sum(dim, p):
    prob = fi.poisson3d_sphere(cells=4, p=p) if dim == 3 else fi.poisson2d_circle(cells=4, p=p)
    prob["geometry"] = dict(kind="none")
    prob["dirichlet"] = dict(kind="none")
    prob["kappa"] = 2.5
    prob["hi"] = tuple(0.7 + 0.1 * a for a in range(dim))   # non-square cells
    K, _, cls = element_system(prob, (1,) * dim)
    assert cls == INSIDE
    hs = [(prob["hi"][a] - prob["lo"][a]) / 4 for a in range(dim)]
    Ks, Ms = zip(*[element_1d_matrices(p, h) for h in hs])
    assert np.allclose(K, 2.5 * kron_sum(Ks, Ms), rtol=0, atol=1e-13)


def test_fictitious_cell_scales_by_alpha():
    prob = fi.poisson2d_circle(cells=16, p=2, alpha=1e-6)
    Kin, _, c1 = element_system(prob, (8, 8))
    Kout, _, c2 = element_system(prob, (0, 0))
    assert (c1, c2) == (INSIDE, OUTSIDE)
    assert np.allclose(Kout, 1e-6 * Kin, rtol=1e-13, atol=1e-15 * np.abs(Kout).max())


def _rigid_modes(p, x0, x1):
    """Translations and rotations interpolated in the hierarchical basis: the
    nodal coefficients are the field values at the corners, bubbles 0 (both
    fields are linear, so this is exact)."""
    from oracle.grid import local_modes
    modes = local_modes(3, p)
    n = len(modes)
    out = []
    fields = [lambda x: (1, 0, 0), lambda x: (0, 1, 0), lambda x: (0, 0, 1),
              lambda x: (0, -x[2], x[1]), lambda x: (x[2], 0, -x[0]), lambda x: (-x[1], x[0], 0)]
    for f in fields:
        v = np.zeros(3 * n)
        for l, js in enumerate(modes):
            if max(js) > 1:
                continue
            x = [x1[a] if js[a] == 1 else x0[a] for a in range(3)]
            u = f(x)
            for k in range(3):
                v[k * n + l] = u[k]
        out.append(v)
    return np.array(out).T


@pytest.mark.parametrize("p", [1, 2])
def test_elasticity_rigid_body_nullspace(p):
    prob = fi.elasticity3d_voids(cells=4, p=p, n_voids=1)
    prob["geometry"] = dict(kind="none")
    prob["dirichlet"] = dict(kind="none")
    prob["traction"] = None
    cell = (1, 2, 1)
    K, _, _ = element_system(prob, cell)
    x0, x1 = cell_box(prob["lo"], prob["hi"], prob["cells"], cell)
    R = _rigid_modes(p, x0, x1)
    assert np.abs(K @ R).max() < 1e-12 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 1e-10 * ev.max()) == 6
    assert np.allclose(K, K.T, atol=1e-15 * np.abs(K).max())


def test_elasticity_matrix():
    C = elasticity_C(2.0, 0.25, 3)
    lam = 2.0 * 0.25 / (1.25 * 0.5)
    mu = 2.0 / 2.5
    # uniaxial strain e_xx = 1: sigma_xx = lam + 2 mu, sigma_yy = lam
    s = C @ np.array([1, 0, 0, 0, 0, 0.0])
    assert np.allclose(s, [lam + 2 * mu, lam, lam, 0, 0, 0])
    s = C @ np.array([0, 0, 0, 0, 0, 1.0])
    assert np.allclose(s, [0, 0, 0, 0, 0, mu])


@pytest.mark.parametrize("make", [
    lambda: fi.poisson2d_circle(cells=8, p=2, alpha=1e-3),
    lambda: fi.poisson3d_sphere(cells=2, p=2, alpha=1e-2),
])
def test_nodal_load_is_weighted_volume(make):
    """sum over nodal DOFs of b = int alpha f dOmega when f = 1 and there is
    no penalty load (g = 0)."""
    prob = make()
    prob["source"] = dict(kind="const", f0=1.0)
    prob["dirichlet"] = dict(kind="levelset", g="zero")
    A, b, cls = assemble(prob)
    d = prob["dim"]
    C = prob["cells"]
    m = m_1d(C[0], prob["p"])
    idx = np.indices((m,) * d).reshape(d, -1)[::-1]   # per-axis 1D index, x fastest
    nodal = np.all(idx <= C[0], axis=0)
    r = prob["geometry"]["radius"]
    vol_phys = math.pi * r * r if d == 2 else 4 / 3 * math.pi * r ** 3
    expect = vol_phys + prob["alpha"] * (1.0 - vol_phys)
    assert abs(b[nodal].sum() - expect) < 3e-3 * expect


@pytest.mark.parametrize("make", [
    lambda: fi.poisson2d_circle(cells=6, p=2),
    lambda: fi.poisson3d_sphere(cells=2, p=2),
    lambda: fi.square_mms(cells=4, p=3),
])
def test_assembled_matrix_spd(make):
    A, b, _ = assemble(make())
    D = A.toarray()
    assert np.allclose(D, D.T, rtol=0, atol=1e-13 * np.abs(D).max())
    np.linalg.cholesky(D)


def _l2_error(prob, x):
    """||u_h - u||_L2 over the whole (body-fitted) square by a 6-point rule."""
    err = 0.0
    for cell in all_cells(prob["dim"], prob["cells"]):
        x0, x1 = cell_box(prob["lo"], prob["hi"], prob["cells"], cell)
        pts, w = leaf_rule(x0, x1, 5)
        N, _ = shape_functions(prob["p"], x0, x1, pts)
        uh = N @ x[cell_dofs(prob["dim"], prob["cells"], prob["p"], cell)]
        err += float(np.sum(w * (uh - exact_solution(prob, pts)) ** 2))
    return math.sqrt(err)


def test_manufactured_solution_h_convergence():
    """Body-fitted square (Sec. 4.1, psi = 0) with a strong penalty: the L2
    error falls like h^(p+1)."""
    for p in (1, 2):
        errs = []
        for C in (4, 8, 16):
            prob = fi.square_mms(cells=C, p=p, beta=1e9)
            A, b, _ = assemble(prob)
            x = spla.spsolve(A.tocsc(), b)
            errs.append(_l2_error(prob, x))
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert rates[-1] > p + 1 - 0.35, (p, errs, rates)


def test_manufactured_solution_p_convergence():
    errs = []
    for p in (1, 2, 3, 4, 5):
        prob = fi.square_mms(cells=4, p=p, beta=1e11)
        A, b, _ = assemble(prob)
        x = spla.spsolve(A.tocsc(), b)
        errs.append(_l2_error(prob, x))
    assert all(errs[i + 1] < errs[i] / 3 for i in range(len(errs) - 1)), errs


def test_immersed_solution_approaches_exact():
    """Immersed sphere with u = sin sin sin: the physical-domain error drops
    under h-refinement (penalty and alpha limit the rate)."""
    errs = []
    for C in (2, 4):
        prob = fi.poisson3d_sphere(cells=C, p=2)
        A, b, _ = assemble(prob)
        x = spla.spsolve(A.tocsc(), b)
        # error at the centre region (well inside the sphere)
        e = 0.0
        for cell in all_cells(3, prob["cells"]):
            x0, x1 = cell_box(prob["lo"], prob["hi"], prob["cells"], cell)
            pts, w = leaf_rule(x0, x1, 4)
            keep = np.linalg.norm(pts - 0.5, axis=1) < 0.3
            if not keep.any():
                continue
            N, _ = shape_functions(2, x0, x1, pts[keep])
            uh = N @ x[cell_dofs(3, prob["cells"], 2, cell)]
            e += float(np.sum(w[keep] * (uh - exact_solution(prob, pts[keep])) ** 2))
        errs.append(math.sqrt(e))
    assert errs[1] < errs[0] / 4, errs


# --------------------------------------------------------------------------
# Linear elasticity (Eq. weakform with the Voigt strain operator B and the
# isotropic C).  Each pin below fails under a plausible slip in the integrand:
# a tensor instead of an engineering shear strain in B (shear energy x 1/4),
# 2 mu on the shear diagonal of C (x 2), a wrong lambda (dilatation energy),
# a traction term left off the load or put on the wrong face.

def _lame_closed_form(E, nu):
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def _interpolate_linear(dim, p, x0, x1, Gm):
    """Coefficients of u(x) = Gm x in the hierarchical basis of one cell:
    the corner values on the nodal modes, zero on the bubbles (exact, since u
    is multilinear), fields stacked."""
    from oracle.grid import local_modes
    modes = local_modes(dim, p)
    n = len(modes)
    v = np.zeros(dim * n)
    for l, js in enumerate(modes):
        if max(js) > 1:
            continue
        x = np.array([x1[a] if js[a] == 1 else x0[a] for a in range(dim)])
        u = Gm @ x
        for k in range(dim):
            v[k * n + l] = u[k]
    return v


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 3), (3, 1), (3, 2)])
def test_elasticity_strain_energy_closed_form(dim, p):
    """1/2 u^T K u of a homogeneous strain u = G x on one uncut cell equals
    the closed-form energy V (lambda/2 (tr eps)^2 + mu eps:eps), eps = sym G
    (plane strain in 2D), for random G and for pure shear, uniaxial strain and
    dilatation separately."""
    E, nu = 3.0, 0.27
    prob = fi.elasticity_mms(dim=dim, cells=3, p=p, E=E, nu=nu)
    prob["dirichlet"] = dict(kind="none")
    prob["hi"] = tuple(0.8 + 0.15 * a for a in range(dim))   # non-cubic cells
    cell = (1,) * dim
    K, _, cls = element_system(prob, cell)
    assert cls == INSIDE
    x0, x1 = cell_box(prob["lo"], prob["hi"], prob["cells"], cell)
    vol = float(np.prod(np.asarray(x1) - np.asarray(x0)))
    lam, mu = _lame_closed_form(E, nu)
    rng = np.random.default_rng(7)
    fields = [rng.uniform(-1, 1, (dim, dim)) for _ in range(3)]
    shear = np.zeros((dim, dim))
    shear[0, 1] = 0.7                                  # u_x = 0.7 y: pure shear
    uni = np.zeros((dim, dim))
    uni[0, 0] = 0.4
    fields += [shear, shear.T, uni, 0.3 * np.eye(dim)]
    if dim == 3:
        for a, b in ((1, 2), (2, 0)):
            g = np.zeros((3, 3))
            g[a, b] = -0.5
            fields.append(g)
    for Gm in fields:
        u = _interpolate_linear(dim, p, x0, x1, Gm)
        eps = 0.5 * (Gm + Gm.T)
        expect = vol * (0.5 * lam * np.trace(eps) ** 2 + mu * np.sum(eps * eps))
        got = 0.5 * u @ K @ u
        assert abs(got - expect) <= 1e-12 * max(1.0, abs(expect)), (Gm, got, expect)


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 1), (3, 2)])
def test_elasticity_displacement_patch_test(dim, p):
    """Patch test: on a 3^d body-fitted block without body force, the
    coefficients of a linear field u = G x prescribed on every mode that is
    nonzero on the boundary (corner values on nodes, 0 on bubbles) give, by
    the interior equations, exactly that field (interior nodes = G x, every
    interior bubble 0)."""
    prob = fi.elasticity_mms(dim=dim, cells=3, p=p)
    prob["source"] = dict(kind="const", f0=0.0)
    prob["dirichlet"] = dict(kind="none")
    prob["hi"] = (1.0, 1.3, 0.9)[:dim]
    A, b, _ = assemble(prob)
    assert np.abs(b).max() == 0.0
    Gm = np.random.default_rng(3).uniform(-1, 1, (dim, dim))
    C = prob["cells"]
    m = [m_1d(C[a], p) for a in range(dim)]
    M = int(np.prod(m))
    idx = np.indices(m[::-1]).reshape(dim, -1)[::-1]   # per-axis 1D index, x fastest
    nodal = np.all([idx[a] <= C[a] for a in range(dim)], axis=0)
    # a mode is nonzero on the box boundary iff along some axis it is an end node
    boundary = np.any([(idx[a] == 0) | (idx[a] == C[a]) for a in range(dim)], axis=0)
    h = [(prob["hi"][a] - prob["lo"][a]) / C[a] for a in range(dim)]
    X = np.array([prob["lo"][a] + h[a] * idx[a] for a in range(dim)])   # node coordinates
    exact = np.zeros(dim * M)
    for k in range(dim):
        exact[k * M:(k + 1) * M] = np.where(nodal, (Gm[k] @ X), 0.0)
    fixed = np.tile(boundary, dim)
    free = ~fixed
    Ad = A.toarray()
    u = exact.copy()
    u[free] = np.linalg.solve(Ad[np.ix_(free, free)], -Ad[np.ix_(free, fixed)] @ exact[fixed])
    assert np.abs(u - exact).max() <= 1e-10 * np.abs(exact).max()


def test_elasticity_traction_resultant():
    """The traction load on a box face is int t N dGamma: tested against a
    constant field (resultant t x face area) and a linear one (first moment)
    per component, on a box with unequal sides; a load on the wrong face or a
    dropped term fails one of them."""
    prob = fi.elasticity_mms(dim=3, cells=2, p=2)
    prob["source"] = dict(kind="const", f0=0.0)
    prob["dirichlet"] = dict(kind="none")
    prob["hi"] = (1.0, 2.0, 3.0)
    t = np.array([0.7, -1.3, 2.1])
    prob["traction"] = dict(face=1, t=tuple(t))        # the face x = 1, area 2 x 3
    _, b, _ = assemble(prob)
    C, p = prob["cells"], prob["p"]
    m = [m_1d(C[a], p) for a in range(3)]
    M = int(np.prod(m))
    idx = np.indices(m[::-1]).reshape(3, -1)[::-1]
    nodal = np.all([idx[a] <= C[a] for a in range(3)], axis=0)
    X = np.array([prob["lo"][a] + (prob["hi"][a] - prob["lo"][a]) / C[a] * idx[a]
                  for a in range(3)])
    for k in range(3):
        bk = b[k * M:(k + 1) * M]
        assert abs(bk[nodal].sum() - t[k] * 6.0) <= 1e-12 * 6.0
        # u = y e_k: int_0^2 int_0^3 y dz dy = 6; u = z e_k: 9; u = x e_k: 6 (x = 1)
        assert abs(bk[nodal] @ X[1][nodal] - t[k] * 6.0) <= 1e-12 * 9.0
        assert abs(bk[nodal] @ X[2][nodal] - t[k] * 9.0) <= 1e-12 * 9.0
        assert abs(bk[nodal] @ X[0][nodal] - t[k] * 6.0) <= 1e-12 * 9.0


def test_elasticity_manufactured_force_is_navier():
    """The oracle's manufactured body force equals -div sigma(u) computed by
    central differences of u with sigma = lambda (div u) I + mu (grad u +
    grad u^T) (no Voigt notation involved)."""
    from oracle.assembly import exact_solution, source_values
    for dim in (2, 3):
        prob = fi.elasticity_mms(dim=dim, E=2.0, nu=0.31)
        lam, mu = _lame_closed_form(2.0, 0.31)
        pts = np.random.default_rng(5).uniform(0.1, 0.9, (6, dim))
        hh = 1e-4

        def sigma(x):
            J = np.empty((dim, dim))              # J[i, j] = d u_i / d x_j
            for j in range(dim):
                e = np.zeros(dim)
                e[j] = hh
                J[:, j] = (exact_solution(prob, (x + e)[None])[0]
                           - exact_solution(prob, (x - e)[None])[0]) / (2 * hh)
            return lam * np.trace(J) * np.eye(dim) + mu * (J + J.T)

        for x in pts:
            div = np.zeros(dim)
            for j in range(dim):
                e = np.zeros(dim)
                e[j] = hh
                div += (sigma(x + e)[:, j] - sigma(x - e)[:, j]) / (2 * hh)
            f = source_values(prob, x[None])[0]
            assert np.allclose(f, -div, rtol=0, atol=2e-5 * np.abs(f).max()), (dim, f, -div)


def _l2_error_vec(prob, x):
    d = prob["dim"]
    M = int(np.prod([m_1d(prob["cells"][a], prob["p"]) for a in range(d)]))
    err = 0.0
    for cell in all_cells(d, prob["cells"]):
        x0, x1 = cell_box(prob["lo"], prob["hi"], prob["cells"], cell)
        pts, w = leaf_rule(x0, x1, prob["p"] + 3)
        N, _ = shape_functions(prob["p"], x0, x1, pts)
        dofs = cell_dofs(d, prob["cells"], prob["p"], cell)
        ex = exact_solution(prob, pts)
        for k in range(d):
            uh = N @ x[k * M + dofs]
            err += float(np.sum(w * (uh - ex[:, k]) ** 2))
    return math.sqrt(err)


@pytest.mark.parametrize("dim,p,cells", [(3, 1, (2, 4, 8)), (3, 2, (2, 4, 6)), (2, 2, (4, 8, 16))])
def test_elasticity_manufactured_h_convergence(dim, p, cells):
    """Body-fitted elasticity with the manufactured displacement
    prod sin(pi x_a) (1, -2, 3): the L2 error falls like h^(p+1).  A wrong
    shear scaling solves another operator, and the error stalls."""
    errs, hs = [], []
    for C in cells:
        prob = fi.elasticity_mms(dim=dim, cells=C, p=p, beta=1e10)
        A, b, _ = assemble(prob)
        x = spla.spsolve(A.tocsc(), b)
        errs.append(_l2_error_vec(prob, x))
        hs.append(1.0 / C)
    rate = math.log(errs[-2] / errs[-1]) / math.log(hs[-2] / hs[-1])
    assert rate > p + 1 - 0.35, (errs, rate)
