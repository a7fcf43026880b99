"""Structured grid and degree-of-freedom layout (oracle).

Test infrastructure only (see ``oracle/__init__``).

Hierarchical DOF ordering (Sec. 3.2, Eq. restrictionoperation): on a
Cartesian grid the tensor-product space Q_p is the tensor product of 1D C0
spaces, so each axis gets its own 1D index with the nodal functions first
and the bubbles of each degree in consecutive blocks:

    node k (k = 0..C)                        -> k
    bubble of degree q (q = 2..p) in cell c  -> (C + 1) + (q - 2) C + c

A level of degree p' uses exactly the 1D indices below m(p') = C p' + 1, so
the DOFs of level l-1 are a prefix sub-box of those of level l and the
restriction R_l = [I 0] is a sub-box selection.  The global index of a
scalar DOF with 1D indices (i_x, i_y, i_z) is i_x + m i_y + m^2 i_z (x
fastest); vector fields (elasticity) stack whole scalar fields,
I = f M + scalar index with M = m^d.

Local numbering inside a cell: 1D local mode j (0 = left node, 1 = right
node, q = bubble of degree q), local index j_x + (p+1) j_y + (p+1)^2 j_z,
fields stacked the same way: l = f (p+1)^d + scalar local index.
"""
from __future__ import annotations

import itertools

import numpy as np


def m_1d(C: int, p: int) -> int:
    """Number of 1D indices per axis at degree p on C cells."""
    return C * p + 1


def dof_1d(C: int, c: int, j: int) -> int:
    """1D index of local mode j of cell c."""
    if j == 0:
        return c
    if j == 1:
        return c + 1
    return (C + 1) + (j - 2) * C + c


def ndofs(dim: int, cells, p: int, nf: int = 1) -> int:
    n = nf
    for a in range(dim):
        n *= m_1d(cells[a], p)
    return n


def cell_dofs(dim: int, cells, p: int, cell, nf: int = 1) -> np.ndarray:
    """Global indices of the (p+1)^d nf DOFs of one cell, in local order."""
    ms = [m_1d(cells[a], p) for a in range(dim)]
    M = int(np.prod(ms))
    per_axis = [[dof_1d(cells[a], cell[a], j) for j in range(p + 1)] for a in range(dim)]
    scalar = []
    # local index j_x + (p+1) j_y + ... : x fastest
    for js in itertools.product(*[range(p + 1)] * dim):
        js = js[::-1]  # itertools varies the last slot fastest; reverse so x is fastest
        g = 0
        stride = 1
        for a in range(dim):
            g += per_axis[a][js[a]] * stride
            stride *= ms[a]
        scalar.append(g)
    scalar = np.array(scalar, dtype=np.int64)
    return np.concatenate([f * M + scalar for f in range(nf)])


def all_cells(dim: int, cells):
    """Cell multi-indices in linear order (x fastest)."""
    for idx in itertools.product(*[range(cells[a]) for a in reversed(range(dim))]):
        yield tuple(reversed(idx))


def cell_linear(dim: int, cells, cell) -> int:
    g = 0
    stride = 1
    for a in range(dim):
        g += cell[a] * stride
        stride *= cells[a]
    return g


def cell_box(lo, hi, cells, cell):
    """Corners of a cell: x0 = lo + c h, x1 = lo + (c+1) h, h = (hi-lo)/C."""
    x0, x1 = [], []
    for a in range(len(cells)):
        h = (hi[a] - lo[a]) / cells[a]
        x0.append(lo[a] + cell[a] * h)
        x1.append(lo[a] + (cell[a] + 1) * h)
    return tuple(x0), tuple(x1)


def local_modes(dim: int, p: int):
    """Per-axis local modes (j_x, j_y, ...) for each scalar local index."""
    out = []
    for js in itertools.product(*[range(p + 1)] * dim):
        out.append(js[::-1])
    return out
