"""Hierarchical multigrid V-cycle and preconditioned CG (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

* Level hierarchy (Sec. 3.2).  The coarse p-levels follow the arithmetic
  p-sequence p, p-1, ..., 1.  Because the basis is hierarchical
  (Eq. hierarchicalFunctions) the restriction is the binary matrix
  R_l = [I 0] of Eq. (restrictionoperation) and the level matrices are the
  corresponding sub-blocks of the fine matrix (Eq. hierarchicalMatrices):
  A_{l-1} = R_l A_l R_l^T.  Below p = 1 the Remark of Sec. 3.2 allows
  standard geometric multigrid; the reading here is nested Q1 grids with
  C -> ceil(C/2) cells per axis, prolongation P = multilinear interpolation,
  restriction P^T and Galerkin coarse matrices P^T A P, until every axis has
  at most `coarse_cells` cells.  The coarsest system is solved directly
  (dense Cholesky), the "exact" solve on level 0 of Algorithm 1.
* Additive Schwarz smoother (Eq. AdditiveSchwarz) with elementwise blocks
  (Sec. 3.3.1): block i holds every DOF supported on cell i,
  A_i = P_i^T A P_i, M^{-1} = sum_i P_i A_i^{-1} P_i^T; or with patchwise
  blocks (Sec. 3.3.1, the grouping the paper uses for multi-level hp grids
  and compares on uniform ones in Sec. 4.1): block v holds every DOF
  supported on the (up to 2^d) cells around mesh node v.  Relaxation
  (Sec. 3.3.2): omega = 1/3 (2D) and 2/15 (3D) elementwise, 1/6 and 1/18
  patchwise, on every level l != 0.  Sec. 3.3.2 derives omega from the
  stability condition rho(I - omega M^{-1} A) < 1, i.e. omega < 2 / lambda_max,
  with lambda_max bounded by the block overlap.  With penalty-dominated cut
  cells lambda_max exceeds 2^d (the supports of elementwise blocks overlap
  3^d times), and the heuristic values break that condition on levels whose
  coarse correction does not remove the offending modes.  Reading: each level
  keeps the paper's omega unless omega * lambda_est > THETA (= 1.75, a margin
  below 2 for the estimate), in which case omega = THETA / lambda_est.
  lambda_est is the A-inner-product Rayleigh quotient after POWER_ITERS steps
  of the power method on M^{-1} A from the start vector v_i = sin(i + 1).
* Comparison smoothers (Sec. 4.1, Table tab:testcaseA): damped Jacobi
  (damping 2/3, not stated in the paper) and symmetric Gauss-Seidel (forward
  sweeps before, backward sweeps after the coarse correction).
* V-cycle: Algorithm 1.  The printed algorithm repeats
  x <- x + omega M^{-1} r without refreshing r; read literally n_s steps
  would collapse into one step with n_s omega.  The reading is that r is
  recomputed as b - A x before every smoothing step (smoothing is a
  fixed-point iteration, Sec. 3.1), which keeps the cycle symmetric.
* PCG (Sec. 4): x_0 = 0, one V-cycle per iteration, stop when the relative
  residual ||b - A x_i|| / ||b|| falls below the tolerance.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assembly import assemble, nfields
from .grid import all_cells, cell_dofs, m_1d


THETA = 1.75
POWER_ITERS = 40


AS_KINDS = ("elementwise", "patchwise")


def default_omega(dim, smoother="elementwise"):
    if smoother == "elementwise":
        return 1.0 / 3.0 if dim == 2 else 2.0 / 15.0
    if smoother == "patchwise":
        return 1.0 / 6.0 if dim == 2 else 1.0 / 18.0
    if smoother == "jacobi":
        return 2.0 / 3.0
    if smoother == "gauss_seidel":
        return 1.0
    raise ValueError(smoother)


def p_selection(dim, cells, p_fine, p_coarse, nf=1):
    """Indices (in the fine level) of the coarse level's DOFs, ordered as
    the coarse level numbers them: the prefix sub-box [0, m(p_coarse))^d."""
    mf = [m_1d(cells[a], p_fine) for a in range(dim)]
    mc = [m_1d(cells[a], p_coarse) for a in range(dim)]
    Mf = int(np.prod(mf))
    ranges = [np.arange(mc[a]) for a in range(dim)]
    grids = np.meshgrid(*ranges, indexing="ij")
    # coarse order: x fastest -> iterate with the last axis slowest
    idx = np.zeros(grids[0].shape, dtype=np.int64)
    stride = 1
    for a in range(dim):
        idx = idx + grids[a] * stride
        stride *= mf[a]
    scalar = idx.transpose(tuple(reversed(range(dim)))).ravel()
    return np.concatenate([f * Mf + scalar for f in range(nf)])


def q1_prolongation_1d(Cf: int) -> np.ndarray:
    """Nodes 0..Cf of a fine 1D grid from the ceil(Cf/2)-cell coarse grid:
    even node 2k = coarse node k, odd node 2k+1 = average of k and k+1."""
    Cc = (Cf + 1) // 2
    P = np.zeros((Cf + 1, Cc + 1))
    for i in range(Cf + 1):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            P[i, i // 2] = 0.5
            P[i, i // 2 + 1] = 0.5
    return P


def q1_prolongation(dim, cells_f, nf=1):
    """Tensor-product Q1 prolongation (x fastest), block diagonal in fields."""
    P = sp.csr_matrix(np.ones((1, 1)))
    for a in reversed(range(dim)):
        P = sp.kron(P, sp.csr_matrix(q1_prolongation_1d(cells_f[a])), format="csr")
    if nf > 1:
        P = sp.kron(sp.identity(nf, format="csr"), P, format="csr")
    return P.tocsr()


class Level:
    def __init__(self, A, cells, p, nf, dim):
        self.A = A.tocsr()
        self.cells = tuple(cells)
        self.p = p
        self.nf = nf
        self.dim = dim
        self.N = A.shape[0]
        self.to_coarse = None   # ("p", selection) or ("h", P)
        self.blocks = None      # explicit additive Schwarz blocks, if given
        self.kind = None        # smoother kind, set with the smoother
        self.IDX = None
        self.Ainv = None
        self.chol = None

    def block_dofs(self, smoother="elementwise"):
        """Global DOF indices of every additive Schwarz block: one block per
        cell (elementwise) or per mesh node (patchwise: the union of the
        cells' DOFs around the node, sorted)."""
        if smoother == "elementwise":
            return [cell_dofs(self.dim, self.cells, self.p, c, self.nf)
                    for c in all_cells(self.dim, self.cells)]
        blocks = []
        for v in itertools.product(*[range(self.cells[a] + 1) for a in reversed(range(self.dim))]):
            v = tuple(reversed(v))  # x fastest
            cs = []
            for off in itertools.product((0, 1), repeat=self.dim):
                c = tuple(v[a] - off[a] for a in range(self.dim))
                if all(0 <= c[a] < self.cells[a] for a in range(self.dim)):
                    cs.append(c)
            blocks.append(np.unique(np.concatenate(
                [cell_dofs(self.dim, self.cells, self.p, c, self.nf) for c in cs])))
        return blocks

    def build_blocks(self, smoother="elementwise"):
        """Additive Schwarz blocks A_i = P_i^T A P_i, inverted through
        their Cholesky factor.  Blocks of equal size are stacked (IDX, Ainv
        for the elementwise case, where all have the same size; `groups`
        holds one (IDX, Ainv) pair per block size)."""
        by_size = {}
        blocks = self.blocks if self.blocks is not None else self.block_dofs(smoother)
        for idx in blocks:
            by_size.setdefault(len(idx), []).append(idx)
        self.groups = []
        for n, lst in sorted(by_size.items()):
            IDX = np.array(lst)
            Ainv = np.empty((len(IDX), n, n))
            for i, idx in enumerate(IDX):
                Ai = self.A[idx][:, idx].toarray()
                L = np.linalg.cholesky(Ai)
                Linv = sla.solve_triangular(L, np.eye(n), lower=True)
                Ainv[i] = Linv.T @ Linv
            self.groups.append((IDX, Ainv))
        if len(self.groups) == 1:
            self.IDX, self.Ainv = self.groups[0]
        else:
            self.IDX = self.Ainv = None

    def build_pointwise(self, smoother):
        """Comparison smoothers of Sec. 4.1: Jacobi (the diagonal) or
        Gauss-Seidel (the lower and upper triangles with the diagonal)."""
        if smoother == "jacobi":
            self.dinv = 1.0 / self.A.diagonal()
        else:
            self.lower = sp.tril(self.A, 0, format="csr")
            self.upper = sp.triu(self.A, 0, format="csr")

    def pre_correction(self, r):
        """Correction of one pre-smoothing step from the residual r:
        omega M^{-1} r (additive Schwarz, Jacobi) or a forward Gauss-Seidel
        sweep (D + L)^{-1} r."""
        if self.kind == "gauss_seidel":
            return spla.spsolve_triangular(self.lower, r, lower=True)
        if self.kind == "jacobi":
            return self.omega * (self.dinv * r)
        return self.omega * self.smoother(r)

    def post_correction(self, r):
        """Post-smoothing: as pre_correction, but a backward Gauss-Seidel
        sweep (D + U)^{-1} r, so that the V-cycle stays symmetric."""
        if self.kind == "gauss_seidel":
            return spla.spsolve_triangular(self.upper, r, lower=False)
        return self.pre_correction(r)

    def lambda_max_estimate(self, iters=POWER_ITERS):
        """Power method on M^{-1} A (self-adjoint in the A inner product):
        returns (v^T A M^{-1} A v) / (v^T A v) after `iters` steps."""
        v = np.sin(np.arange(self.N, dtype=np.float64) + 1.0)
        lam = 0.0
        for _ in range(iters):
            Av = self.A @ v
            w = self.smoother(Av)
            lam = (Av @ w) / (v @ Av)
            v = w / np.linalg.norm(w)
        return lam

    def smoother(self, r):
        """M^{-1} r = sum_i P_i A_i^{-1} P_i^T r."""
        z = np.zeros(self.N)
        for IDX, Ainv in self.groups:
            Z = np.einsum("bij,bj->bi", Ainv, r[IDX])
            z += np.bincount(IDX.ravel(), weights=Z.ravel(), minlength=self.N)
        return z


class Hierarchy:
    """Multigrid levels 0 (coarsest, direct) .. L (the given system)."""

    def __init__(self, prob, A=None, b=None, omega=None):
        if A is None:
            A, b, _ = assemble(prob)
        self._configure(prob, b, omega)
        d = prob["dim"]
        nf = nfields(prob)
        cells = tuple(prob["cells"])
        levels = [Level(A, cells, prob["p"], nf, d)]
        # arithmetic p-sequence
        for pc in range(prob["p"] - 1, 0, -1):
            fine = levels[-1]
            sel = p_selection(d, cells, fine.p, pc, nf)
            fine.to_coarse = ("p", sel)
            levels.append(Level(fine.A[sel][:, sel], cells, pc, nf, d))
        self._complete(levels)

    def _configure(self, prob, b, omega):
        self.prob = prob
        self.b = b
        self.smoother_kind = prob.get("smoother", "elementwise")
        self.omega = omega if omega is not None else (
            prob["omega"] if prob.get("omega") is not None
            else default_omega(prob["dim"], self.smoother_kind))
        self.n_pre = prob["n_pre"]
        self.n_post = prob["n_post"]

    def _complete(self, levels):
        """Append the nested Q1 h-levels below `levels` (ordered fine to
        coarse, the last one a Q1 level of the base grid in grid order),
        then build the smoothers and the coarse factor."""
        prob = self.prob
        d = prob["dim"]
        nf = nfields(prob)
        # nested Q1 h-levels
        cmax = prob["coarse_cells"]
        while max(levels[-1].cells) > cmax:
            fine = levels[-1]
            P = q1_prolongation(d, fine.cells, nf)
            fine.to_coarse = ("h", P)
            Ac = (P.T @ fine.A @ P).tocsr()
            cc = tuple((c + 1) // 2 for c in fine.cells)
            levels.append(Level(Ac, cc, 1, nf, d))
        levels.reverse()
        self.levels = levels
        self._setup_smoothers()
        c = levels[0]
        c.chol = sla.cho_factor(c.A.toarray(), lower=True)

    def _setup_smoothers(self):
        """Per level l != 0: additive Schwarz blocks with omega clamped by
        the stability reading, or a comparison smoother (Jacobi with the
        damping 2/3, symmetric Gauss-Seidel without damping)."""
        for lv in self.levels[1:]:
            lv.kind = self.smoother_kind
            if self.smoother_kind in AS_KINDS:
                lv.build_blocks(self.smoother_kind)
                lv.lam = lv.lambda_max_estimate()
                lv.omega = min(self.omega, THETA / lv.lam)
            else:
                lv.build_pointwise(self.smoother_kind)
                lv.omega = self.omega

    def _complete_on_nodes(self, levels, nodes):
        """As _complete, for a last level that holds only the base-grid
        nodes `nodes` (grid node ids, x fastest; fully fictitious cells
        removed): Q1 h-levels by Galerkin P^T A P with P = multilinear
        interpolation onto the held fine nodes, coarse nodes that no held
        fine node depends on dropped; then smoothers and coarse Cholesky."""
        d, nf = levels[-1].dim, levels[-1].nf
        cells = levels[-1].cells
        while max(levels[-1].cells) > self.prob["coarse_cells"]:
            fine = levels[-1]
            P = q1_prolongation(d, cells, 1)[nodes]
            used = np.flatnonzero(np.asarray(abs(P).sum(axis=0)).ravel() > 0)
            P = P[:, used]
            if nf > 1:
                P = sp.kron(sp.identity(nf, format="csr"), P, format="csr")
            fine.to_coarse = ("h", P.tocsr())
            cells = tuple((c + 1) // 2 for c in cells)
            lv = Level((P.T @ fine.A @ P).tocsr(), cells, 1, nf, d)
            lv.blocks = self._q1_blocks(cells, used, nf)
            levels.append(lv)
            nodes = used
        levels.reverse()
        self.levels = levels
        self._setup_smoothers()
        levels[0].chol = sla.cho_factor(levels[0].A.toarray(), lower=True)

    def _q1_blocks(self, cells, nodes, nf):
        """Blocks of a Q1 level holding grid nodes `nodes`: the held nodes
        of each cell (elementwise) or of the cells around each node."""
        d = len(cells)
        pos = {int(n): i for i, n in enumerate(nodes)}
        M = len(nodes)

        def cell_nodes(c):
            out = []
            for off in itertools.product((0, 1), repeat=d):
                g, stride = 0, 1
                for a in range(d):
                    g += (c[a] + off[a]) * stride
                    stride *= cells[a] + 1
                if g in pos:
                    out.append(pos[g])
            return out

        def fields(ids):
            ids = np.unique(np.array(ids, dtype=np.int64))
            return np.concatenate([f * M + ids for f in range(nf)])

        blocks = []
        if self.smoother_kind == "elementwise":
            for c in all_cells(d, cells):
                ids = cell_nodes(c)
                if ids:
                    blocks.append(fields(ids))
            return blocks
        for v in itertools.product(*[range(cells[a] + 1) for a in reversed(range(d))]):
            v = tuple(reversed(v))
            ids = [i for c in cells_around(v, cells) for i in cell_nodes(c)]
            if ids:
                blocks.append(fields(ids))
        return blocks

    @property
    def A(self):
        return self.levels[-1].A

    def restrict(self, l, r):
        kind, op = self.levels[l].to_coarse
        return r[op] if kind == "p" else op.T @ r

    def prolong_add(self, l, x, xc):
        kind, op = self.levels[l].to_coarse
        if kind == "p":
            x[op] += xc
        else:
            x += op @ xc
        return x

    def vcycle(self, b, l=None):
        """x = V(b) with zero initial guess on level l (Algorithm 1)."""
        if l is None:
            l = len(self.levels) - 1
        lv = self.levels[l]
        if l == 0:
            return sla.cho_solve(lv.chol, b)
        x = np.zeros_like(b)
        for s in range(self.n_pre):
            r = b - lv.A @ x
            x = x + lv.pre_correction(r)
        r = b - lv.A @ x
        xc = self.vcycle(self.restrict(l, r), l - 1)
        x = self.prolong_add(l, x, xc)
        for s in range(self.n_post):
            r = b - lv.A @ x
            x = x + lv.post_correction(r)
        return x


def pcg(A, b, precond, rtol=1e-8, maxit=500, flexible=False, x0=None):
    """Preconditioned conjugate gradients from x_0 = 0 (Sec. 4).

    Returns (x, iterations, relres history).  The iteration count is the
    number of search directions used when ||r_k|| / ||b|| <= rtol first
    holds for the recursively updated residual; the true residual is then
    checked and the iteration continues from it if it is not below rtol.
    `flexible` uses the Polak-Ribiere form beta = r_{k+1}^T (z_{k+1} - z_k)
    / r_k^T z_k, which tolerates a preconditioner that is not exactly
    symmetric."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = precond(r)
    p = z.copy()
    rz = r @ z
    k = 0
    while k < maxit:
        k += 1
        q = A @ p
        a = rz / (p @ q)
        x = x + a * p
        r = r - a * q
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if rel <= rtol:
            rt = b - A @ x
            if np.linalg.norm(rt) / nb <= rtol:
                return x, k, hist
            r = rt
        zn = precond(r)
        rzn = r @ zn
        beta = (rzn - r @ z) / rz if flexible else rzn / rz
        z = zn
        rz = rzn
        p = z + beta * p
    return x, k, hist


def mg_solve(A, b, vcycle, rtol=1e-9, maxit=500):
    """Multigrid as a stand-alone solver, x_{i+1} = x_i + V(b - A x_i),
    with the contraction numbers rho_i = ||r_i|| / ||r_{i-1}|| of Sec. 4.
    A diverging iteration (the residual grown 1e20-fold) stops early; the
    caller sees it in the returned residual history."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    norms = [np.linalg.norm(r)]
    k = 0
    while norms[-1] / nb > rtol and k < maxit:
        if not norms[-1] <= 1e20 * nb:
            break
        k += 1
        with np.errstate(over="ignore", invalid="ignore"):
            x = x + vcycle(r)
            r = b - A @ x
        norms.append(np.linalg.norm(r))
    rho = [norms[i] / norms[i - 1] for i in range(1, len(norms))]
    return x, k, rho


def solve(prob, rtol=1e-8, maxit=500, flexible=False):
    """Assemble, build the hierarchy and run V-cycle PCG."""
    H = Hierarchy(prob)
    x, k, hist = pcg(H.A, H.b, H.vcycle, rtol=rtol, maxit=maxit, flexible=flexible)
    return H, x, k, hist


def cells_around(v, C):
    """The (up to 2^d) cells of a grid with C cells per axis around node v."""
    d = len(C)
    out = []
    for off in itertools.product((0, 1), repeat=d):
        c = tuple(v[a] - off[a] for a in range(d))
        if all(0 <= c[a] < C[a] for a in range(d)):
            out.append(c)
    return out
