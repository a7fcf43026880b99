"""Multi-level hp overlays and their hp-multigrid (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

Mesh (Sec. 2.2).  Level 0 is the base grid of C_1 x ... x C_d cells.  An
element of level k that is refined is overlaid by its 2^d bisection children,
the elements of level k+1, recursively up to the depth K.  Refinement follows
the geometry, as in the examples of Sec. 4.2 and 4.3 where elements cut by
the immersed boundary are refined to a predefined depth: an element is
refined when ``geometry.classify_box`` calls it cut.  Leaf elements are the
elements without children.  Level k is the uniform lattice of C_a 2^k cells
per axis; element (k, e) is lattice cell e of it.

Basis.  Every element of every level carries the (p+1)^d tensor-product
integrated Legendre modes of ``oracle.basis`` on its own box, with the same
p on all levels.  A mode (j_1, ..., j_d) of element e belongs to the
topological component of the level-k lattice with doubled coordinates
t_a = 2 e_a (j_a = 0), 2 e_a + 2 (j_a = 1) or 2 e_a + 1 (bubble, j_a >= 2):
a vertex when every t_a is even, otherwise an edge, face or interior with one
bubble degree per odd axis.  The elements of level k whose closure contains
the component share its functions, which are C0 across them.  A function of
an element is a polynomial on that element's box; on every leaf below it it
is evaluated at the mapped points, so a leaf's element matrix couples the
functions of all its ancestors (refinement by superposition).  With
trunk-space elements (``MlhpSpace(trunk=True)``, the space of ``oracle.trunk``)
a component keeps only the bubble-degree combinations that sum to at most p.

Activation.  The paper defers the rule set to Zander et al.; the reading
here is one that makes the active functions a basis of exactly the C0 space
of piecewise Q_p functions on the leaf elements (checked by brute force in
the tests):

  R1 compatibility: a component of level k >= 1 on the boundary of the
     refined zone Z_k (the union of the level-k elements; faces of the box
     do not count) is inactive, so overlay functions vanish where an overlay
     meets unrefined elements.  Test: some in-box lattice cell of level k
     whose closure contains the component is not an element.
  R2 hats: a vertex of level k >= 1 at the position of a level k-1 vertex
     (every lattice node index even) is inactive; the coarser hat is there.
  R3 high order: the functions of an edge, face or interior of level k are
     active only if the component belongs to at least one leaf element; the
     high-order modes of refined elements are represented by their children.

Numbering.  Fields outermost (I = f M + s, as on uniform grids); the scalar
functions are ordered by level, then by component (last axis slowest, x
fastest), then by bubble degrees (first odd axis fastest).  On the base grid
the vertices therefore come in the node order of the uniform Q1 grid.

hp-multigrid (Sec. 3.2, Fig. hpmultigrid).  The polynomial degree is lowered
first on all elements: level p_l keeps the functions whose bubble degrees are
all at most p_l (vertices have degree 1).  At p = 1 the overlays are then
removed from the finest down (drop the hats of level k), which leaves the Q1
space of the base grid.  Each step keeps a subset of the functions, so the
restriction is a binary selection and the coarse matrix the principal
sub-matrix of the fine one (Eq. restrictionoperation, Eq. hierarchicalMatrices).
Below the base grid the nested Q1 h-levels and the Cholesky coarse solve of
``oracle.multigrid`` follow.

Additive Schwarz blocks (Sec. 3.3.1, Fig. patchBlocks).  A function touches
the base cells that contain an element of its support.  Patchwise block v:
every function touching one of the (up to 2^d) base cells around base node v.
Elementwise block c: every function touching base cell c (the grouping at the
granularity of base elements).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .assembly import (boundary_faces, dirichlet_values, mass_terms, nfields,
                       shape_functions, volume_terms)
from .geometry import CUT, INSIDE, OUTSIDE, classify_box
from .grid import all_cells, local_modes
from .multigrid import Hierarchy, Level, pcg
from .quadrature import cell_rules, face_rule, leaf_rule


def _rev(t):
    return tuple(reversed(t))


def mode_position(e_a: int, j: int) -> int:
    """Doubled lattice coordinate of 1D local mode j of cell e_a."""
    if j == 0:
        return 2 * e_a
    if j == 1:
        return 2 * e_a + 2
    return 2 * e_a + 1


class MlhpMesh:
    """Elements E[k] and refined elements R[k] of every level k = 0..K."""

    def __init__(self, dim, cells, lo, hi, depth, refine):
        """refine(k, e, x0, x1) -> bool decides whether element (k, e) with
        box [x0, x1] is overlaid by children (only asked for k < depth)."""
        self.dim = dim
        self.cells = tuple(cells)
        self.lo = tuple(lo)
        self.hi = tuple(hi)
        self.depth = depth
        self.E = [set(all_cells(dim, self.cells))]
        self.R = []
        for k in range(depth):
            Rk = {e for e in self.E[k] if refine(k, e, *self.box(k, e))}
            self.R.append(Rk)
            kids = set()
            for e in Rk:
                for off in itertools.product((0, 1), repeat=dim):
                    kids.add(tuple(2 * e[a] + off[a] for a in range(dim)))
            self.E.append(kids)
        self.R.append(set())

    def lattice(self, k, a):
        return self.cells[a] << k

    def box(self, k, e):
        x0, x1 = [], []
        for a in range(self.dim):
            h = (self.hi[a] - self.lo[a]) / self.lattice(k, a)
            x0.append(self.lo[a] + e[a] * h)
            x1.append(self.lo[a] + (e[a] + 1) * h)
        return tuple(x0), tuple(x1)

    def elements(self, k):
        return sorted(self.E[k], key=_rev)

    def leaves(self):
        return [(k, e) for k in range(self.depth + 1)
                for e in sorted(self.E[k] - self.R[k], key=_rev)]

    def ancestors(self, k, e):
        """(j, index) of the element's ancestors j = 0..k (itself last)."""
        return [(j, tuple(ea >> (k - j) for ea in e)) for j in range(k + 1)]

    def neighbours(self, k, t):
        """In-box lattice cells of level k whose closure contains component t."""
        ranges = []
        for a in range(self.dim):
            if t[a] % 2:
                ranges.append([(t[a] - 1) // 2])
            else:
                n = self.lattice(k, a)
                ranges.append([c for c in (t[a] // 2 - 1, t[a] // 2) if 0 <= c < n])
        return list(itertools.product(*ranges))

    def active(self, k, t) -> bool:
        """Activation rules R1-R3 of the module docstring."""
        nb = self.neighbours(k, t)
        Ek = self.E[k]
        if k >= 1 and not all(c in Ek for c in nb):
            return False                                        # R1
        if all(ta % 2 == 0 for ta in t):
            return not (k >= 1 and all(ta % 4 == 0 for ta in t))  # R2
        return any(c in Ek and c not in self.R[k] for c in nb)  # R3

    def locate(self, x):
        """Leaf (k, e) whose box contains point x (upper faces belong to the
        lower cell at the end of the box)."""
        k = 0
        while True:
            e = []
            for a in range(self.dim):
                n = self.lattice(k, a)
                h = (self.hi[a] - self.lo[a]) / n
                e.append(min(n - 1, max(0, int((x[a] - self.lo[a]) // h))))
            e = tuple(e)
            if e in self.R[k]:
                k += 1
                continue
            assert e in self.E[k]
            return k, e


class MlhpSpace:
    """Active functions of a multi-level hp mesh at degree p; with
    trunk=True only the modes whose bubble degrees sum to at most p
    (trunk-space elements, as ``oracle.trunk`` defines them)."""

    def __init__(self, mesh: MlhpMesh, p: int, nf: int = 1, trunk: bool = False):
        self.mesh = mesh
        self.p = p
        self.nf = nf
        self.trunk = trunk
        d = mesh.dim
        self.modes = local_modes(d, p)
        comps = {}
        for k in range(mesh.depth + 1):
            for e in mesh.elements(k):
                for js in self.modes:
                    t = tuple(mode_position(e[a], js[a]) for a in range(d))
                    if (k, t) not in comps:
                        comps[(k, t)] = mesh.active(k, t)
        keys = sorted((kt for kt, on in comps.items() if on),
                      key=lambda kt: (kt[0], _rev(kt[1])))
        funcs = []
        for k, t in keys:
            odd = [a for a in range(d) if t[a] % 2]
            for qs in itertools.product(range(2, p + 1), repeat=len(odd)):
                if trunk and sum(qs) > p:
                    continue
                funcs.append((k, t, _rev(qs)))
        self.funcs = funcs
        self.fid = {f: i for i, f in enumerate(funcs)}
        self.M = len(funcs)
        self.N = nf * self.M
        self.level = np.array([f[0] for f in funcs], dtype=np.int64)
        # polynomial degree of each function's mode: the largest bubble degree,
        # or for trunk elements their sum (level p_l keeps degree <= p_l)
        agg = sum if trunk else max
        self.degree = np.array([agg(f[2]) if f[2] else 1 for f in funcs], dtype=np.int64)

    def restrict(self, keep):
        """Keep only the functions where `keep` (a mask over the present
        ones) is true, renumbered in their order (removal of the functions
        that only fully fictitious leaves support)."""
        self.funcs = [f for f, k in zip(self.funcs, keep) if k]
        self.fid = {f: i for i, f in enumerate(self.funcs)}
        self.M = len(self.funcs)
        self.N = self.nf * self.M
        self.level = self.level[keep]
        self.degree = self.degree[keep]
        self._touch = None

    def leaf_functions(self, k, e):
        """Per ancestor j of leaf (k, e): (j, box, active local-mode columns
        of its (p+1)^d modes, their scalar function ids)."""
        d = self.mesh.dim
        out = []
        for j, ae in self.mesh.ancestors(k, e):
            cols, ids = [], []
            for m, js in enumerate(self.modes):
                t = tuple(mode_position(ae[a], js[a]) for a in range(d))
                qs = tuple(js[a] for a in range(d) if t[a] % 2)
                f = self.fid.get((j, t, qs))
                if f is not None:
                    cols.append(m)
                    ids.append(f)
            out.append((j, self.mesh.box(j, ae), np.array(cols, dtype=np.int64),
                        np.array(ids, dtype=np.int64)))
        return out

    def eval_on_leaf(self, k, e, pts, funcs=None):
        """Scalar functions supported on leaf (k, e) at points:
        (ids (n,), N (Q, n), grad N (Q, n, d))."""
        if funcs is None:
            funcs = self.leaf_functions(k, e)
        ids, Ns, Gs = [], [], []
        for _, (x0, x1), cols, fids in funcs:
            if len(cols) == 0:
                continue
            N, G = shape_functions(self.p, x0, x1, pts)
            ids.append(fids)
            Ns.append(N[:, cols])
            Gs.append(G[:, cols])
        return np.concatenate(ids), np.concatenate(Ns, axis=1), np.concatenate(Gs, axis=1)

    def dofs(self, ids):
        """Field-major global DOFs of scalar functions `ids`."""
        return np.concatenate([f * self.M + ids for f in range(self.nf)])

    def touched_base_cells(self):
        """Per scalar function: the base cells that contain an element of its
        support (as linear base-cell indices, x fastest)."""
        if getattr(self, "_touch", None) is not None:
            return self._touch
        mesh = self.mesh
        C = mesh.cells
        out = []
        for k, t, _ in self.funcs:
            s = set()
            for c in mesh.neighbours(k, t):
                if c in mesh.E[k]:
                    b = tuple(ca >> k for ca in c)
                    lin, stride = 0, 1
                    for a in range(mesh.dim):
                        lin += b[a] * stride
                        stride *= C[a]
                    s.add(lin)
            out.append(sorted(s))
        self._touch = out
        return out

    def evaluate(self, coef, pts):
        """Scalar field sum_i coef_i N_i at points (first field only)."""
        vals = np.empty(len(pts))
        for q, x in enumerate(np.atleast_2d(pts)):
            k, e = self.mesh.locate(x)
            ids, N, _ = self.eval_on_leaf(k, e, x[None, :])
            vals[q] = N[0] @ coef[ids]
        return vals


def mesh_for(prob) -> MlhpMesh:
    """The overlay mesh of a problem: depth prob['overlay_levels'], elements
    refined where prob.get('refine_geometry', prob['geometry']) cuts them,
    or by a callable prob['refine'](k, e, x0, x1)."""
    rule = prob.get("refine")
    if rule is None:
        geom = prob.get("refine_geometry", prob["geometry"])

        def rule(k, e, x0, x1):
            return classify_box(geom, x0, x1) == CUT
    return MlhpMesh(prob["dim"], prob["cells"], prob["lo"], prob["hi"],
                    prob.get("overlay_levels", 0), rule)


def _leaf_faces(prob, mesh, k, e):
    return boundary_faces(prob, e, tuple(mesh.lattice(k, a) for a in range(mesh.dim)))


def outside_base_cells(mesh: MlhpMesh, geom) -> set:
    """Base cells lying wholly outside the physical domain."""
    return {e for e in mesh.E[0] if classify_box(geom, *mesh.box(0, e)) == OUTSIDE}


def kept_functions(space: MlhpSpace, geom) -> np.ndarray:
    """Removal of fully fictitious cells on an overlay mesh, at the
    granularity of base cells: a function is kept iff it touches a base
    cell that is not wholly outside (boolean mask over the scalar
    functions).  Removing single overlay leaves instead would leave
    functions that are linearly dependent on the remaining leaves (a
    singular system); overlay leaves inside kept base cells stay, weighted
    by alpha."""
    mesh = space.mesh
    C = mesh.cells
    out = set()
    for e in outside_base_cells(mesh, geom):
        lin, stride = 0, 1
        for a in range(mesh.dim):
            lin += e[a] * stride
            stride *= C[a]
        out.add(lin)
    return np.array([any(c not in out for c in cs) for cs in space.touched_base_cells()])


def leaf_system(prob, space: MlhpSpace, k, e):
    """(scalar ids, K_L, b_L, class) of leaf (k, e): the terms of
    Eq. (weakform) integrated over the leaf's box with the space tree of
    ``oracle.quadrature`` (cut leaves) or one tensor Gauss rule."""
    mesh = space.mesh
    p = space.p
    x0, x1 = mesh.box(k, e)
    cls = classify_box(prob["geometry"], x0, x1)
    if cls == CUT:
        vp, vw, va, spts, sw = cell_rules(prob, x0, x1)
    else:
        vp, vw = leaf_rule(x0, x1, p)
        va = np.full(len(vw), 1.0 if cls == INSIDE else prob["alpha"])
        spts, sw = np.zeros((0, mesh.dim)), np.zeros(0)
    funcs = space.leaf_functions(k, e)
    ids, N, G = space.eval_on_leaf(k, e, vp, funcs)
    K, b = volume_terms(prob, N, G, vp, vw, va)
    beta = prob["beta"]
    if len(sw):
        _, Ns, _ = space.eval_on_leaf(k, e, spts, funcs)
        Ms, bs = mass_terms(prob, Ns, sw, dirichlet_values(prob, spts))
        K = K + beta * Ms
        b = b + beta * bs
    for face, kind in _leaf_faces(prob, mesh, k, e):
        fp, fw = face_rule(x0, x1, face, p)
        _, Nf, _ = space.eval_on_leaf(k, e, fp, funcs)
        if kind == "D":
            Ms, bs = mass_terms(prob, Nf, fw, dirichlet_values(prob, fp))
            K = K + beta * Ms
            b = b + beta * bs
        else:
            t = np.array(prob["traction"]["t"][: prob["dim"]])
            _, bt = mass_terms(prob, Nf, fw, np.tile(t, (len(fw), 1)))
            b = b + bt
    return ids, K, b, cls


def assemble_mlhp(prob, space: MlhpSpace = None):
    """Global CSR matrix and load over the active functions, summed from the
    leaf element systems.  Returns (A, b, space)."""
    drop = bool(prob.get("drop_outside"))
    if space is None:
        space = MlhpSpace(mesh_for(prob), prob["p"], nfields(prob),
                          trunk=prob.get("space", "tensor") == "trunk")
        if drop:
            space.restrict(kept_functions(space, prob["geometry"]))
    rows, cols, vals = [], [], []
    b = np.zeros(space.N)
    removed = outside_base_cells(space.mesh, prob["geometry"]) if drop else set()
    for k, e in space.mesh.leaves():
        if k == 0 and e in removed:
            continue
        ids, K, bl, _ = leaf_system(prob, space, k, e)
        dofs = space.dofs(ids)
        rows.append(np.repeat(dofs, len(dofs)))
        cols.append(np.tile(dofs, len(dofs)))
        vals.append(K.ravel())
        np.add.at(b, dofs, bl)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(space.N, space.N)).tocsr()
    A.sum_duplicates()
    return A, b, space


def hp_level_sets(space: MlhpSpace):
    """Scalar function ids of every hp-multigrid level, fine to coarse: the
    degrees p, p-1, ..., 1, then at p = 1 the overlays K, K-1, ..., 1
    removed; the last set is the base grid's hats.  Sets equal to the one
    before them (an overlay level without active hats) are skipped."""
    sets = [np.arange(space.M)]
    for pc in range(space.p - 1, 0, -1):
        sets.append(np.flatnonzero(space.degree <= pc))
    hats = space.degree == 1
    for kk in range(space.mesh.depth, 0, -1):
        s = np.flatnonzero(hats & (space.level < kk))
        if len(s) != len(sets[-1]):
            sets.append(s)
    return sets


def schwarz_blocks(space, members, kind):
    """Additive Schwarz blocks of the level holding scalar functions
    `members` (positions in that level, fields expanded): one per base cell
    (elementwise) or per base node (patchwise), x fastest."""
    mesh = space.mesh
    d = mesh.dim
    C = mesh.cells
    pos = -np.ones(space.M, dtype=np.int64)
    pos[members] = np.arange(len(members))
    touch = space.touched_base_cells()
    per_cell = [[] for _ in range(int(np.prod(C)))]
    for f in members:
        for c in touch[f]:
            per_cell[c].append(pos[f])
    Ml = len(members)

    def fields(ids):
        ids = np.array(sorted(set(ids)), dtype=np.int64)
        return np.concatenate([f * Ml + ids for f in range(space.nf)])

    if kind == "elementwise":
        return [fields(lst) for lst in per_cell]
    blocks = []
    for v in itertools.product(*[range(C[a] + 1) for a in reversed(range(d))]):
        v = _rev(v)
        ids = []
        for off in itertools.product((0, 1), repeat=d):
            c = tuple(v[a] - off[a] for a in range(d))
            if all(0 <= c[a] < C[a] for a in range(d)):
                lin, stride = 0, 1
                for a in range(d):
                    lin += c[a] * stride
                    stride *= C[a]
                ids += per_cell[lin]
        blocks.append(fields(ids))
    return blocks


class MlhpHierarchy(Hierarchy):
    """hp-multigrid on a multi-level hp mesh (Sec. 3.2), followed by the
    nested Q1 h-levels of the base grid and the coarse Cholesky."""

    def __init__(self, prob, omega=None):
        A, b, space = assemble_mlhp(prob)
        self.space = space
        if "smoother" not in prob:
            prob = dict(prob, smoother="patchwise")
        self._configure(prob, b, omega)
        d = prob["dim"]
        nf = space.nf
        sets = hp_level_sets(space)
        self.level_sets = sets
        fine_sel = sets[0]
        levels = [Level(A, tuple(prob["cells"]), space.p, nf, d)]
        levels[0].blocks = schwarz_blocks(space, sets[0], self.smoother_kind)
        for s in sets[1:]:
            fine = levels[-1]
            where = np.searchsorted(fine_sel, s)
            Mf = len(fine_sel)
            sel = np.concatenate([f * Mf + where for f in range(nf)])
            fine.to_coarse = ("p", sel)
            lv = Level(fine.A[sel][:, sel], tuple(prob["cells"]),
                       int(space.degree[s].max()), nf, d)
            lv.blocks = schwarz_blocks(space, s, self.smoother_kind)
            levels.append(lv)
            fine_sel = s
        if prob.get("drop_outside"):
            # the last set holds the kept base-grid hats: continue on those nodes
            C = space.mesh.cells
            nodes = []
            for f in fine_sel:
                _, t, _ = space.funcs[f]
                g, stride = 0, 1
                for a in range(d):
                    g += (t[a] // 2) * stride
                    stride *= C[a] + 1
                nodes.append(g)
            self._complete_on_nodes(levels, np.array(nodes, dtype=np.int64))
        else:
            self._complete(levels)


def mlhp_solve(prob, rtol=1e-8, maxit=500):
    """Assemble on the overlay mesh, build the hp-multigrid and run PCG."""
    H = MlhpHierarchy(prob)
    x, k, hist = pcg(H.A, H.b, H.vcycle, rtol=rtol, maxit=maxit)
    return H, x, k, hist
