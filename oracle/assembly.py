"""Element matrices and global assembly of the FCM system (oracle).

Test infrastructure only (see ``oracle/__init__``).

Discrete weak form of the finite cell method (Sec. 2.1, Eq. weakform):

  a(u, v) = int (B v)^T alpha C B u dOmega + int beta (N v)^T N u dGamma_D
  b(v)    = int alpha (N v)^T f dOmega + int (N v)^T g_N dGamma_N
            + int beta (N v)^T g_D dGamma_D

For the Poisson problem B = grad and C = kappa; for elasticity B is the
Voigt strain operator and C the isotropic elasticity matrix.  The global
matrix is assembled in CSR form from per-cell matrices in the layout of
``oracle.grid``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .basis import basis_1d
from .geometry import CUT, INSIDE, classify_box, rotated_coordinates
from .grid import all_cells, cell_box, cell_dofs, local_modes, ndofs
from .quadrature import cell_rules, face_rule, leaf_rule


def nfields(prob):
    return prob["dim"] if prob["pde"] == "elasticity" else 1


def shape_functions(p, x0, x1, pts):
    """Scalar tensor-product modes at physical points of the cell [x0, x1].
    Returns N (Q, n) and grad N (Q, n, d)."""
    pts = np.atleast_2d(pts)
    d = pts.shape[1]
    vals, ders = [], []
    for a in range(d):
        xi = (2.0 * pts[:, a] - (x0[a] + x1[a])) / (x1[a] - x0[a])
        Na, dNa = basis_1d(p, xi)
        vals.append(Na)
        ders.append(dNa * (2.0 / (x1[a] - x0[a])))
    modes = np.array(local_modes(d, p))          # (n, d)
    N = np.ones((pts.shape[0], len(modes)))
    for a in range(d):
        N = N * vals[a][modes[:, a]].T
    G = np.empty((pts.shape[0], len(modes), d))
    for b in range(d):
        g = np.ones_like(N)
        for a in range(d):
            tab = ders[a] if a == b else vals[a]
            g = g * tab[modes[:, a]].T
        G[:, :, b] = g
    return N, G


def elasticity_C(E, nu, d):
    """Isotropic elasticity matrix in Voigt notation."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    if d == 3:
        C = np.zeros((6, 6))
        C[:3, :3] = lam
        for i in range(3):
            C[i, i] += 2.0 * mu
        for i in range(3, 6):
            C[i, i] = mu
        return C
    C = np.zeros((3, 3))  # plane strain
    C[:2, :2] = lam
    C[0, 0] += 2.0 * mu
    C[1, 1] += 2.0 * mu
    C[2, 2] = mu
    return C


def strain_B(G):
    """Voigt strain operator at each point: (Q, nv, d n), field-major
    columns (all u_x modes, then u_y, then u_z)."""
    Q, n, d = G.shape
    if d == 3:
        B = np.zeros((Q, 6, 3 * n))
        gx, gy, gz = G[:, :, 0], G[:, :, 1], G[:, :, 2]
        B[:, 0, 0:n] = gx
        B[:, 1, n:2 * n] = gy
        B[:, 2, 2 * n:3 * n] = gz
        B[:, 3, n:2 * n] = gz
        B[:, 3, 2 * n:3 * n] = gy
        B[:, 4, 0:n] = gz
        B[:, 4, 2 * n:3 * n] = gx
        B[:, 5, 0:n] = gy
        B[:, 5, n:2 * n] = gx
        return B
    B = np.zeros((Q, 3, 2 * n))
    gx, gy = G[:, :, 0], G[:, :, 1]
    B[:, 0, 0:n] = gx
    B[:, 1, n:2 * n] = gy
    B[:, 2, 0:n] = gy
    B[:, 2, n:2 * n] = gx
    return B


def source_values(prob, pts):
    """Body load f at points (Poisson: scalar; elasticity: (Q, d))."""
    s = prob["source"]
    d = prob["dim"]
    if prob["pde"] == "elasticity":
        if s["kind"] == "elastic_sin3":
            return _elastic_sin3_force(prob, pts)
        return np.zeros((len(pts), d)) + s.get("f0", 0.0)
    if s["kind"] == "const":
        return np.full(len(pts), float(s["f0"]))
    if s["kind"] == "sin3":
        u = np.ones(len(pts))
        for a in range(d):
            u = u * np.sin(math.pi * pts[:, a])
        return prob["kappa"] * d * math.pi ** 2 * u
    if s["kind"] == "square_mms":
        a = s["a"]
        if s.get("angle", 0.0) != 0.0:
            xp, yp = rotated_coordinates((0.5, 0.5), s["angle"], pts)
            return np.cos(a * xp) * np.sin(a * yp)
        return np.cos(a * (pts[:, 0] - 0.5)) * np.sin(a * (pts[:, 1] - 0.5))
    if s["kind"] == "popcorn":
        # f = -kappa Lap u for u = x^3 + x y^2 + y^3 + z^4 + sin(3 (x^2 + y^2))
        x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
        r2 = x * x + y * y
        lap = 8.0 * x + 6.0 * y + 12.0 * z * z + 12.0 * np.cos(3.0 * r2) - 36.0 * r2 * np.sin(3.0 * r2)
        return -prob["kappa"] * lap
    raise ValueError(s["kind"])


def _lame(E, nu):
    """Lame parameters (lambda, mu) of an isotropic material."""
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def _elastic_sin3_force(prob, pts):
    """Body force of the manufactured displacement u = phi(x) v with
    phi = prod_a sin(pi x_a) and a constant vector v (plane strain in 2D):
    Navier's equation -div sigma = f with sigma = lambda (div u) I + 2 mu eps
    gives f = -(mu Lap u + (lambda + mu) grad div u)
           = mu d pi^2 phi v - (lambda + mu) H(phi) v,
    H the Hessian of phi: H_aa = -pi^2 phi,
    H_ab = pi^2 cos(pi x_a) cos(pi x_b) prod_{c != a, b} sin(pi x_c)."""
    d = prob["dim"]
    v = np.asarray(prob["source"]["v"][:d], dtype=float)
    lam, mu = _lame(prob["E"], prob["nu"])
    sn = np.sin(math.pi * pts)
    cs = np.cos(math.pi * pts)
    phi = np.prod(sn, axis=1)
    H = np.empty((len(pts), d, d))
    for a in range(d):
        for b in range(d):
            if a == b:
                H[:, a, a] = -math.pi ** 2 * phi
            else:
                t = math.pi ** 2 * cs[:, a] * cs[:, b]
                for c in range(d):
                    if c != a and c != b:
                        t = t * sn[:, c]
                H[:, a, b] = t
    return mu * d * math.pi ** 2 * phi[:, None] * v[None, :] - (lam + mu) * (H @ v)


def dirichlet_values(prob, pts):
    """Prescribed g_D at points (Poisson scalar; elasticity (Q, d))."""
    g = prob["dirichlet"].get("g", "zero")
    d = prob["dim"]
    if prob["pde"] == "elasticity":
        return np.zeros((len(pts), d))
    if g == "zero":
        return np.zeros(len(pts))
    if g == "sin3":
        u = np.ones(len(pts))
        for a in range(d):
            u = u * np.sin(math.pi * pts[:, a])
        return u
    if g == "square_mms":
        s = prob["source"]
        a = s["a"]
        if s.get("angle", 0.0) != 0.0:
            xp, yp = rotated_coordinates((0.5, 0.5), s["angle"], pts)
            return np.cos(a * xp) * np.sin(a * yp) / (2.0 * s["kappa"] * a * a)
        return (np.cos(a * (pts[:, 0] - 0.5)) * np.sin(a * (pts[:, 1] - 0.5))
                / (2.0 * s["kappa"] * a * a))
    if g == "popcorn":
        x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
        return x ** 3 + x * y * y + y ** 3 + z ** 4 + np.sin(3.0 * (x * x + y * y))
    raise ValueError(g)


def exact_solution(prob, pts):
    """Manufactured solution, where the problem has one."""
    s = prob["source"]["kind"]
    if s == "elastic_sin3":
        v = np.asarray(prob["source"]["v"][:prob["dim"]], dtype=float)
        return np.prod(np.sin(math.pi * pts), axis=1)[:, None] * v[None, :]
    if s == "sin3":
        u = np.ones(len(pts))
        for a in range(prob["dim"]):
            u = u * np.sin(math.pi * pts[:, a])
        return u
    if s in ("square_mms", "popcorn"):
        return dirichlet_values(prob, pts)
    raise ValueError("no manufactured solution")


def _volume_terms(prob, x0, x1, pts, w, alpha):
    N, G = shape_functions(prob["p"], x0, x1, pts)
    return volume_terms(prob, N, G, pts, w, alpha)


def volume_terms(prob, N, G, pts, w, alpha):
    """Stiffness and load of one integration domain from the scalar shape
    functions N (Q, n) and their gradients G (Q, n, d) at its points."""
    wa = w * alpha
    f = source_values(prob, pts)
    if prob["pde"] == "poisson":
        K = np.zeros((G.shape[1], G.shape[1]))
        for a in range(G.shape[2]):
            K = K + G[:, :, a].T @ (wa[:, None] * G[:, :, a])
        K = prob["kappa"] * K
        b = N.T @ (wa * f)
        return K, b
    d = prob["dim"]
    Bm = strain_B(G)
    C = elasticity_C(prob["E"], prob["nu"], d)
    CB = np.einsum("vw,qwj->qvj", C, Bm)
    K = np.einsum("qvi,qvj->ij", Bm * wa[:, None, None], CB, optimize=True)
    b = np.concatenate([N.T @ (wa * f[:, k]) for k in range(d)])
    return K, b


def _mass_terms(prob, x0, x1, pts, w, g):
    """beta-free surface mass matrix and load: (int N N^T, int g N)."""
    N, _ = shape_functions(prob["p"], x0, x1, pts)
    return mass_terms(prob, N, w, g)


def mass_terms(prob, N, w, g):
    """Surface mass matrix and load from the scalar shape functions N (Q, n)."""
    Ms = N.T @ (w[:, None] * N)
    nf = nfields(prob)
    if nf == 1:
        return Ms, N.T @ (w * g)
    n = Ms.shape[0]
    M = np.zeros((nf * n, nf * n))
    for k in range(nf):
        M[k * n:(k + 1) * n, k * n:(k + 1) * n] = Ms
    bb = np.concatenate([N.T @ (w * g[:, k]) for k in range(nf)])
    return M, bb


def boundary_faces(prob, cell, cells=None):
    """Box faces of this cell that carry Dirichlet (kind 'D') or traction
    ('T') data: list of (face id, kind).  `cells`: cells per axis of the
    lattice the cell index refers to (default: the problem's grid)."""
    out = []
    d = prob["dim"]
    C = prob["cells"] if cells is None else cells
    dirf = prob["dirichlet"].get("faces", []) if prob["dirichlet"]["kind"] == "faces" else []
    tr = prob.get("traction")
    for a in range(d):
        for s in (0, 1):
            face = 2 * a + s
            on = (cell[a] == 0) if s == 0 else (cell[a] == C[a] - 1)
            if not on:
                continue
            if face in dirf:
                out.append((face, "D"))
            if tr is not None and tr["face"] == face:
                out.append((face, "T"))
    return out


def element_system(prob, cell):
    """(K_c, b_c, class) of one cell: volume terms by the space tree, the
    immersed penalty surface, and box-face penalty and traction terms."""
    lo, hi, C = prob["lo"], prob["hi"], prob["cells"]
    x0, x1 = cell_box(lo, hi, C, cell)
    cls = classify_box(prob["geometry"], x0, x1)
    if cls == CUT:
        vp, vw, va, sp_, sw = cell_rules(prob, x0, x1)
    else:
        vp, vw = leaf_rule(x0, x1, prob["p"])
        va = np.full(len(vw), 1.0 if cls == INSIDE else prob["alpha"])
        sp_, sw = np.zeros((0, len(x0))), np.zeros(0)
    K, b = _volume_terms(prob, x0, x1, vp, vw, va)
    beta = prob["beta"]
    if len(sw):
        Ms, bs = _mass_terms(prob, x0, x1, sp_, sw, dirichlet_values(prob, sp_))
        K = K + beta * Ms
        b = b + beta * bs
    for face, kind in boundary_faces(prob, cell):
        fp, fw = face_rule(x0, x1, face, prob["p"])
        if kind == "D":
            Ms, bs = _mass_terms(prob, x0, x1, fp, fw, dirichlet_values(prob, fp))
            K = K + beta * Ms
            b = b + beta * bs
        else:
            t = np.array(prob["traction"]["t"][: prob["dim"]])
            g = np.tile(t, (len(fw), 1))
            _, bt = _mass_terms(prob, x0, x1, fp, fw, g)
            b = b + bt
    return K, b, cls


def classify_cells(prob):
    """Class of every cell in linear order (x fastest)."""
    lo, hi, C = prob["lo"], prob["hi"], prob["cells"]
    return np.array([classify_box(prob["geometry"], *cell_box(lo, hi, C, c))
                     for c in all_cells(prob["dim"], C)], dtype=np.int8)


def assemble(prob):
    """Global CSR matrix A, load b and per-cell classes of the top level."""
    d, C, p = prob["dim"], prob["cells"], prob["p"]
    nf = nfields(prob)
    N = ndofs(d, C, p, nf)
    rows, cols, vals = [], [], []
    b = np.zeros(N)
    classes = []
    for cell in all_cells(d, C):
        K, bc, cls = element_system(prob, cell)
        dofs = cell_dofs(d, C, p, cell, nf)
        rows.append(np.repeat(dofs, len(dofs)))
        cols.append(np.tile(dofs, len(dofs)))
        vals.append(K.ravel())
        np.add.at(b, dofs, bc)
        classes.append(cls)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A, b, np.array(classes, dtype=np.int8)
