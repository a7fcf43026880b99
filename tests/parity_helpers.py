"""Parity helpers shared by the GPU parity tests (test infrastructure; they
use the oracle only).

* PhysField: the relative L2 norm over the physical domain of the field of a
  coefficient vector, the reading of "relative L2 error" for solutions.
* Noise: the oracle's V-cycle and smoothers with every block inverse taken
  from an LU factorisation instead of Cholesky, the noise floor of two
  backward-stable FP64 computations of the same ill-conditioned operators.
* uniform_index: the uniform-grid number of every function of an
  overlay-free multi-level hp space.
"""
import numpy as np
import scipy.sparse as sp

from oracle.assembly import nfields, shape_functions
from oracle.geometry import INSIDE, OUTSIDE, classify_box
from oracle.grid import all_cells, cell_box, cell_dofs, m_1d, ndofs
from oracle.quadrature import cell_rules, leaf_rule


class PhysField:
    """L2 norm over the physical domain of the field of a coefficient vector:
    quadrature points of the oracle's rules (space tree on cut cells) with
    alpha = 1, shape functions evaluated once per case."""

    def __init__(self, prob):
        d, C, p = prob["dim"], prob["cells"], prob["p"]
        nf = nfields(prob)
        M = ndofs(d, C, p)
        rows, cols, vals, w = [], [], [], []
        q = 0
        for cell in all_cells(d, C):
            x0, x1 = cell_box(prob["lo"], prob["hi"], C, cell)
            c = classify_box(prob["geometry"], x0, x1)
            if c == OUTSIDE:
                continue
            if c == INSIDE:
                pts, wt = leaf_rule(x0, x1, p + 1)
                keep = np.ones(len(wt), dtype=bool)
            else:
                pts, wt, a, _, _ = cell_rules(prob, x0, x1)
                keep = a == 1.0
            if not keep.any():
                continue
            N, _ = shape_functions(p, x0, x1, pts[keep])
            dofs = cell_dofs(d, C, p, cell)
            for f in range(nf):
                qq = q + np.arange(N.shape[0])
                rows.append(np.repeat(qq, N.shape[1]))
                cols.append(np.tile(f * M + dofs, N.shape[0]))
                vals.append(N.ravel())
                w.append(wt[keep])
                q += N.shape[0]
        self.E = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                                                        np.concatenate(cols))),
                               shape=(q, nf * M))
        self.w = np.concatenate(w)

    def norm(self, x):
        v = self.E @ x
        return float(np.sqrt(self.w @ (v * v)))

    def rel(self, a, b):
        return self.norm(a - b) / self.norm(b)


def lu_groups(lv):
    """The level's block inverses recomputed through LU (np.linalg.inv)."""
    out = []
    for IDX, _ in lv.groups:
        B = np.empty((len(IDX), IDX.shape[1], IDX.shape[1]))
        for i, idx in enumerate(IDX):
            B[i] = np.linalg.inv(lv.A[idx][:, idx].toarray())
        out.append((IDX, B))
    return out


class Noise:
    """Oracle V-cycle and smoothers with LU block inverses (the noise floor
    of two backward-stable FP64 computations of the same operators)."""

    def __init__(self, H):
        self.H = H
        self.lu = [None] + [lu_groups(lv) for lv in H.levels[1:]]

    def _swap(self):
        for lv, g in zip(self.H.levels[1:], self.lu[1:]):
            lv.groups, g[:] = list(g), list(lv.groups)

    def vcycle(self, r):
        self._swap()
        try:
            return self.H.vcycle(r)
        finally:
            self._swap()

    def smoother(self, l, x):
        self._swap()
        try:
            return self.H.levels[l].smoother(x)
        finally:
            self._swap()


def uniform_index(space):
    """Uniform-grid scalar index of every function of an overlay-free
    multi-level hp space (oracle.mlhp.MlhpSpace): vertex hats first on the
    (C + 1)-lattice, then per axis the edge modes of degree q grouped by q,
    as oracle.grid numbers the 1D functions."""
    mesh, p = space.mesh, space.p
    C = mesh.cells
    out = []
    for k, t, qs in space.funcs:
        assert k == 0
        g, stride, qi = 0, 1, 0
        for a in range(mesh.dim):
            if t[a] % 2 == 0:
                i = t[a] // 2
            else:
                i = (C[a] + 1) + (qs[qi] - 2) * C[a] + (t[a] - 1) // 2
                qi += 1
            g += i * stride
            stride *= m_1d(C[a], p)
        out.append(g)
    return np.array(out)
