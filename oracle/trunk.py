"""Trunk-space elements and removal of fully fictitious cells (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

The paper's 3D examples use hexahedral trunk-space elements (Sec. 4.3,
Fig. Cube4HolesConv; sizes in Table tab::upperbound) instead of the full
tensor-product space.  With the integrated Legendre modes of
``oracle.basis`` a tensor mode of a cell has, per axis, a nodal mode or a
bubble of degree q in 2..p.  The trunk space of degree p keeps the modes
whose bubble degrees sum to at most p: all vertex and edge modes, the face
modes with q_1 + q_2 <= p and the interior modes with q_1 + q_2 + q_3 <= p
(the classical trunk space of Szabo and Babuska, as cited by the paper
through Duster et al.).  Since the rule is the same on every cell, the
trunk space is a mask on the hierarchical tensor layout of ``oracle.grid``;
its DOFs keep their tensor order and are renumbered consecutively.  Lowering
p keeps a subset, so the p-multigrid transfers stay binary (Sec. 3.2).

Removal of fully fictitious cells (the paper's DOF counts, Sec. 4.3 and
4.3.2, imply it): cells classified outside the physical domain are dropped
together with the DOFs supported only on them.  The nested Q1 h-levels
below p = 1 then interpolate onto the kept fine nodes only, and coarse nodes
that no kept fine node depends on are dropped.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .assembly import element_system, nfields
from .geometry import OUTSIDE
from .grid import all_cells, cell_dofs, local_modes, m_1d, ndofs
from .multigrid import Hierarchy, Level, cells_around


def mode_degrees_1d(C: int, p: int) -> np.ndarray:
    """Per 1D index of a C-cell axis at degree p: 0 for a node, q for a
    bubble of degree q."""
    out = np.zeros(m_1d(C, p), dtype=np.int64)
    for q in range(2, p + 1):
        out[(C + 1) + (q - 2) * C:(C + 1) + (q - 1) * C] = q
    return out


def trunk_local_mask(dim: int, p: int, q_max: int = None) -> np.ndarray:
    """Local modes (x fastest) of the trunk space of degree q_max (default
    p) inside the (p+1)^d tensor modes: bubble degrees sum to <= q_max, none
    above q_max."""
    q_max = p if q_max is None else q_max
    keep = []
    for js in local_modes(dim, p):
        qs = [j for j in js if j >= 2]
        keep.append(sum(qs) <= q_max and all(q <= q_max for q in qs))
    return np.array(keep)


def trunk_global_mask(dim, cells, p, q_max=None) -> np.ndarray:
    """Scalar tensor DOFs (x fastest) that belong to the trunk space."""
    q_max = p if q_max is None else q_max
    deg = [mode_degrees_1d(cells[a], p) for a in range(dim)]
    grids = np.meshgrid(*deg, indexing="ij")            # axis a varies along dim a
    s = np.zeros(grids[0].shape, dtype=np.int64)
    mx = np.zeros(grids[0].shape, dtype=np.int64)
    for g in grids:
        s += g
        mx = np.maximum(mx, g)
    keep = (s <= q_max) & (mx <= q_max)
    return keep.transpose(tuple(reversed(range(dim)))).ravel()   # x fastest


class TrunkSpace:
    """Global numbering of the trunk space on a uniform grid, optionally
    without the fully fictitious cells."""

    def __init__(self, prob, classes=None):
        d, C, p = prob["dim"], tuple(prob["cells"]), prob["p"]
        self.dim, self.cells, self.p = d, C, p
        self.nf = nfields(prob)
        self.Mt = ndofs(d, C, p)                         # scalar tensor DOFs
        keep = trunk_global_mask(d, C, p)
        self.local = trunk_local_mask(d, p)
        self.cell_list = list(all_cells(d, C))
        if prob.get("drop_outside") and classes is not None:
            kept = np.asarray(classes) != OUTSIDE
            self.cell_list = [c for c, k in zip(self.cell_list, kept) if k]
            keep &= _supported(d, C, p, np.flatnonzero(kept))
        self.tensor_index = np.flatnonzero(keep)        # kept scalar tensor DOFs, in order
        self.M = len(self.tensor_index)
        self.N = self.nf * self.M
        self.renumber = -np.ones(self.Mt, dtype=np.int64)
        self.renumber[self.tensor_index] = np.arange(self.M)

    def cell_dofs(self, cell):
        """(local positions in the tensor element matrix, global DOFs) of a
        cell's trunk modes, fields stacked."""
        sc = cell_dofs(self.dim, self.cells, self.p, cell)[self.local]
        n = len(self.local)
        pos = np.concatenate([f * n + np.flatnonzero(self.local) for f in range(self.nf)])
        g = self.renumber[sc]
        assert (g >= 0).all()
        return pos, np.concatenate([f * self.M + g for f in range(self.nf)])


def _supported(dim, C, p, cells) -> np.ndarray:
    """Scalar tensor DOFs supported on at least one of the given cells
    (linear cell ids, x fastest): every local mode of every cell, with the
    1D index of mode j of cell c being c (j = 0), c + 1 (j = 1) or
    (C + 1) + (j - 2) C + c (bubble of degree j)."""
    coords, rem = [], np.asarray(cells, dtype=np.int64)
    for a in range(dim):
        coords.append(rem % C[a])
        rem = rem // C[a]
    used = np.zeros(ndofs(dim, C, p), dtype=bool)
    for js in local_modes(dim, p):
        g = np.zeros(len(cells), dtype=np.int64)
        stride = 1
        for a in range(dim):
            c, j = coords[a], js[a]
            ia = c if j == 0 else (c + 1 if j == 1 else (C[a] + 1) + (j - 2) * C[a] + c)
            g += ia * stride
            stride *= m_1d(C[a], p)
        used[g] = True
    return used


def assemble_trunk(prob):
    """Global CSR matrix and load of the trunk space: each cell's tensor
    element system restricted to its trunk modes.  Returns (A, b, space,
    classes of all cells)."""
    cells = list(all_cells(prob["dim"], prob["cells"]))
    systems = [element_system(prob, c) for c in cells]
    classes = np.array([s[2] for s in systems], dtype=np.int8)
    space = TrunkSpace(prob, classes)
    kept = set(space.cell_list)
    rows, cols, vals = [], [], []
    b = np.zeros(space.N)
    for c, (K, bc, _) in zip(cells, systems):
        if c not in kept:
            continue
        pos, g = space.cell_dofs(c)
        rows.append(np.repeat(g, len(g)))
        cols.append(np.tile(g, len(g)))
        vals.append(K[np.ix_(pos, pos)].ravel())
        np.add.at(b, g, bc[pos])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(space.N, space.N)).tocsr()
    A.sum_duplicates()
    return A, b, space, classes


class TrunkHierarchy(Hierarchy):
    """p-multigrid over trunk spaces p, p-1, ..., 1 (binary selections),
    then the nested Q1 h-levels and the coarse Cholesky of
    ``oracle.multigrid``, restricted to the kept nodes when fully fictitious
    cells are removed."""

    def __init__(self, prob, omega=None):
        A, b, space, _ = assemble_trunk(prob)
        self.space = space
        self._configure(prob, b, omega)
        d, C, nf, p = space.dim, space.cells, space.nf, space.p
        deg = [mode_degrees_1d(C[a], p) for a in range(d)]
        levels = [Level(A, C, p, nf, d)]
        level_t = [space.tensor_index]      # scalar tensor ids held by each level
        for pc in range(p - 1, 0, -1):
            kept_t = level_t[-1]
            qsum = np.zeros(len(kept_t), dtype=np.int64)
            qmax = np.zeros(len(kept_t), dtype=np.int64)
            rem = kept_t.copy()
            for a in range(d):
                m = m_1d(C[a], p)
                qa = deg[a][rem % m]
                rem //= m
                qsum += qa
                qmax = np.maximum(qmax, qa)
            where = np.flatnonzero((qsum <= pc) & (qmax <= pc))
            fine = levels[-1]
            Ml = len(kept_t)
            sel = np.concatenate([f * Ml + where for f in range(nf)])
            fine.to_coarse = ("p", sel)
            levels.append(Level(fine.A[sel][:, sel], C, pc, nf, d))
            level_t.append(kept_t[where])
        for lv, ts in zip(levels, level_t):
            lv.blocks = self._p_blocks(ts)
        nodes = self._q1_nodes(level_t[-1])
        self._complete_on_nodes(levels, nodes)

    def _q1_nodes(self, kept_t):
        """Grid node ids (x fastest) of the p = 1 DOFs (vertices)."""
        d, C, p = self.space.dim, self.space.cells, self.space.p
        out = np.zeros(len(kept_t), dtype=np.int64)
        rem = kept_t.copy()
        stride = 1
        for a in range(d):
            m = m_1d(C[a], p)
            ia = rem % m
            rem //= m
            assert (ia <= C[a]).all()
            out += ia * stride
            stride *= C[a] + 1
        return out

    def _p_blocks(self, ts):
        """Blocks of a p-level holding scalar tensor ids `ts`: the level's
        DOFs of each kept cell (elementwise) or of the kept cells around
        each grid node (patchwise)."""
        sp_ = self.space
        d, C = sp_.dim, sp_.cells
        pos = -np.ones(sp_.Mt, dtype=np.int64)
        pos[ts] = np.arange(len(ts))
        Ml = len(ts)
        kept_cells = set(sp_.cell_list)

        def dofs_of(c):
            sc = cell_dofs(d, C, sp_.p, c)
            return pos[sc[pos[sc] >= 0]]

        def fields(ids):
            ids = np.unique(ids)
            return np.concatenate([f * Ml + ids for f in range(sp_.nf)])

        if self.smoother_kind == "elementwise":
            return [fields(dofs_of(c)) for c in sp_.cell_list]
        blocks = []
        for v in itertools.product(*[range(C[a] + 1) for a in reversed(range(d))]):
            v = tuple(reversed(v))
            ids = [dofs_of(c) for c in cells_around(v, C) if c in kept_cells]
            if ids:
                blocks.append(fields(np.concatenate(ids)))
        return blocks
