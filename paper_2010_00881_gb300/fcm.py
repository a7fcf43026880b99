"""Thin ctypes binding of the C ABI in include/fcm.h.

Argument marshalling only: problem dicts (see ``fcm_inputs``) become the C
descriptors, torch CUDA tensors are passed by data pointer, and every step
of the discretisation and the solve runs in libfcm.so.  There is no CPU
fallback: loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfcm.so")

FCM_OK, FCM_E_INVALID, FCM_E_OOM, FCM_E_CUDA, FCM_E_UNSUPPORTED = 0, 1, 2, 3, 4
FCM_E_NOT_CONVERGED, FCM_E_BREAKDOWN, FCM_E_TIMEOUT = 5, 6, 7
FCM_FP64, FCM_MIXED = 0, 1
GEOM = {"none": 0, "ball": 1, "voids": 2, "ellipsoid": 3, "popcorn": 4}
PDE = {"poisson": 0, "elasticity": 1}
SRC = {"const": 0, "sin3": 1, "square_mms": 2, "popcorn": 3}
DIR = {"none": 0, "levelset": 1, "faces": 2}
GVAL = {"zero": 0, "sin3": 1, "square_mms": 2, "popcorn": 3}
OP_APPLY, OP_SMOOTHER, OP_RESTRICT, OP_PROLONG, OP_COARSE = 0, 1, 2, 3, 4
SMOOTHER = {"elementwise": 0, "patchwise": 1, "jacobi": 2}
METHOD_CG_MG, METHOD_MG, METHOD_CG_AS = 0, 1, 2
SPACE_TENSOR, SPACE_TRUNK = 0, 1
QUAD_POINTS, QUAD_SUMFACT = 0, 1

EXPORTS = ["fcm_setup", "fcm_ndofs", "fcm_rhs", "fcm_apply", "fcm_vcycle", "fcm_num_levels",
           "fcm_level_info_get", "fcm_level_op", "fcm_cell_classes", "fcm_pcg_solve",
           "fcm_pcg_solve_host", "fcm_profile_op", "fcm_op_bytes", "fcm_cell_apply_noalloc",
           "fcm_setup_batch", "fcm_batch_size", "fcm_batch_handle", "fcm_pcg_solve_batch",
           "fcm_batch_destroy", "fcm_destroy", "fcm_last_error", "fcm_dof_layout",
           "fcm_cell_dofs", "fcm_mlhp_create", "fcm_mlhp_destroy", "fcm_mlhp_sizes",
           "fcm_mlhp_functions", "fcm_mlhp_leaves", "fcm_mlhp_patches",
           "fcm_mlhp_leaf_classes", "fcm_mlhp_levels", "fcm_mlhp_restriction_1d",
           "fcm_measure_fma_peak", "fcm_solve", "fcm_mlhp_op_create", "fcm_mlhp_op_ndofs",
           "fcm_mlhp_op_apply", "fcm_mlhp_op_rhs", "fcm_mlhp_op_destroy", "fcm_mlhp_op_prepare",
           "fcm_mlhp_op_level", "fcm_mlhp_op_vcycle", "fcm_mlhp_op_pcg"]


class fcm_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("cells", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("p", C.c_int), ("overlay_levels", C.c_int),
                ("overlay_p", C.c_int), ("space", C.c_int), ("drop_outside", C.c_int)]


class fcm_geometry(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_params", C.c_int), ("params", C.POINTER(C.c_double)),
                ("complement", C.c_int)]


class fcm_physics(C.Structure):
    _fields_ = [("pde", C.c_int), ("kappa", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double), ("source", C.c_int),
                ("f0", C.c_double), ("src_a", C.c_double), ("dirichlet", C.c_int),
                ("g", C.c_int), ("dirichlet_faces", C.c_uint), ("traction_face", C.c_int),
                ("traction", C.c_double * 3), ("quad_depth", C.c_int),
                ("quadrature", C.c_int)]


class fcm_solver_opts(C.Structure):
    _fields_ = [("smoother", C.c_int), ("omega", C.c_double), ("n_pre", C.c_int),
                ("n_post", C.c_int), ("coarse_cells", C.c_int), ("build_mixed", C.c_int)]


class fcm_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("relres_recursive", C.c_double),
                ("relres_true", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("ndofs", C.c_longlong),
                ("kernel_launches", C.c_longlong), ("bytes_moved_est", C.c_longlong),
                ("setup_phase_ms", C.c_double * 5)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["setup_phase_ms"] = list(self.setup_phase_ms)
        return d


class fcm_level_info(C.Structure):
    _fields_ = [("cells", C.c_int * 3), ("p", C.c_int), ("is_h_level", C.c_int),
                ("ndofs", C.c_longlong), ("nloc", C.c_int), ("n_own_cells", C.c_int),
                ("n_own_blocks", C.c_int), ("n_fp64_blocks", C.c_int), ("omega", C.c_double),
                ("lambda_est", C.c_double), ("max_block_cond", C.c_double),
                ("fp64_in_mixed", C.c_int), ("kron_operator", C.c_int),
                ("ndofs_active", C.c_longlong)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["cells"] = tuple(self.cells)
        return d


_lib = None


def load():
    """Load libfcm.so (built by paper_2010_00881_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2010_00881_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.fcm_setup.argtypes = [C.POINTER(fcm_grid), C.POINTER(fcm_geometry), C.POINTER(fcm_physics),
                              C.POINTER(fcm_solver_opts), P, C.POINTER(P)]
    lib.fcm_ndofs.argtypes = [P, C.POINTER(C.c_longlong)]
    lib.fcm_rhs.argtypes = [P, P]
    lib.fcm_apply.argtypes = [P, P, P, C.c_int]
    lib.fcm_vcycle.argtypes = [P, P, P, C.c_int]
    lib.fcm_num_levels.argtypes = [P, C.POINTER(C.c_int)]
    lib.fcm_level_info_get.argtypes = [P, C.c_int, C.POINTER(fcm_level_info)]
    lib.fcm_level_op.argtypes = [P, C.c_int, C.c_int, P, P]
    lib.fcm_cell_classes.argtypes = [P, P]
    lib.fcm_pcg_solve.argtypes = [P, P, P, C.c_double, C.c_int, C.c_int, C.POINTER(fcm_info)]
    lib.fcm_pcg_solve_host.argtypes = [P, P, P, C.c_double, C.c_int, C.c_int, C.POINTER(fcm_info)]
    lib.fcm_profile_op.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
    lib.fcm_op_bytes.argtypes = [P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_longlong)]
    lib.fcm_cell_apply_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int), C.c_int, P, P, P, P]
    lib.fcm_measure_fma_peak.argtypes = [C.c_int, C.POINTER(C.c_double)]
    lib.fcm_solve.argtypes = [P, C.c_int, P, P, C.c_double, C.c_int, C.c_int,
                              C.POINTER(fcm_info), P]
    lib.fcm_setup_batch.argtypes = [C.c_int, C.POINTER(fcm_grid), C.POINTER(fcm_geometry),
                                    C.POINTER(fcm_physics), C.POINTER(fcm_solver_opts), C.c_int, P,
                                    C.POINTER(P)]
    lib.fcm_batch_size.argtypes = [P, C.POINTER(C.c_int)]
    lib.fcm_batch_handle.argtypes = [P, C.c_int, C.POINTER(P)]
    lib.fcm_pcg_solve_batch.argtypes = [P, C.POINTER(P), C.c_double, C.c_int, C.c_int, C.c_int,
                                        C.POINTER(fcm_info)]
    lib.fcm_batch_destroy.argtypes = [P]
    lib.fcm_batch_destroy.restype = None
    lib.fcm_destroy.argtypes = [P]
    lib.fcm_destroy.restype = None
    lib.fcm_dof_layout.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int)]
    lib.fcm_cell_dofs.argtypes = [C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_longlong,
                                  C.POINTER(C.c_longlong)]
    LL = C.POINTER(C.c_longlong)
    IP = C.POINTER(C.c_int)
    lib.fcm_mlhp_create.argtypes = [C.POINTER(fcm_grid), C.POINTER(fcm_geometry), C.POINTER(P)]
    lib.fcm_mlhp_destroy.argtypes = [P]
    lib.fcm_mlhp_destroy.restype = None
    lib.fcm_mlhp_sizes.argtypes = [P, LL, LL, LL, LL]
    lib.fcm_mlhp_functions.argtypes = [P, IP, IP, IP]
    lib.fcm_mlhp_leaves.argtypes = [P, IP, IP, LL, LL]
    lib.fcm_mlhp_patches.argtypes = [P, LL, LL]
    lib.fcm_mlhp_leaf_classes.argtypes = [P, C.POINTER(C.c_byte)]
    lib.fcm_mlhp_levels.argtypes = [P, IP, IP]
    lib.fcm_mlhp_restriction_1d.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
    lib.fcm_mlhp_op_create.argtypes = [P, C.POINTER(fcm_grid), C.POINTER(fcm_geometry),
                                       C.POINTER(fcm_physics), P, C.POINTER(P)]
    lib.fcm_mlhp_op_ndofs.argtypes = [P, LL]
    lib.fcm_mlhp_op_apply.argtypes = [P, P, P]
    lib.fcm_mlhp_op_rhs.argtypes = [P, P]
    lib.fcm_mlhp_op_destroy.argtypes = [P]
    lib.fcm_mlhp_op_destroy.restype = None
    lib.fcm_mlhp_op_prepare.argtypes = [P, C.POINTER(fcm_solver_opts)]
    lib.fcm_mlhp_op_level.argtypes = [P, C.c_int, LL, C.POINTER(C.c_double), IP, IP]
    lib.fcm_mlhp_op_vcycle.argtypes = [P, P, P]
    lib.fcm_mlhp_op_pcg.argtypes = [P, P, P, C.c_double, C.c_int, C.POINTER(fcm_info)]
    lib.fcm_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("fcm_destroy", "fcm_batch_destroy", "fcm_last_error", "fcm_mlhp_destroy",
                        "fcm_mlhp_op_destroy"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class FcmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fcm status {status}: {msg}")
        self.status = status


def _check(st, allow=()):
    if st != FCM_OK and st not in allow:
        raise FcmError(st, load().fcm_last_error().decode())
    return st


def dof_layout(cells: int, p: int) -> np.ndarray:
    """1D index of local mode j of cell c on one axis: map[c, j]."""
    out = np.empty(cells * (p + 1), dtype=np.int32)
    _check(load().fcm_dof_layout(cells, p, out.ctypes.data_as(C.POINTER(C.c_int))))
    return out.reshape(cells, p + 1)


def cell_dofs(dim: int, cells, p: int, nf: int, cell: int) -> np.ndarray:
    """Global indices of the DOFs of one cell (linear index, x fastest)."""
    cs = (C.c_int * 3)(*(list(cells) + [1] * (3 - len(cells))))
    out = np.empty(nf * (p + 1) ** dim, dtype=np.int64)
    _check(load().fcm_cell_dofs(dim, cs, p, nf, cell,
                                out.ctypes.data_as(C.POINTER(C.c_longlong))))
    return out


class Overlay:
    """Multi-level hp overlay topology of a problem dict, built on the host
    by the library (fcm_mlhp_*); no GPU is involved."""

    def __init__(self, prob: dict):
        g, gm, _, _, self._keep = descriptors(prob)
        lib = load()
        h = C.c_void_p()
        _check(lib.fcm_mlhp_create(C.byref(g), C.byref(gm), C.byref(h)))
        try:
            n = [C.c_longlong() for _ in range(4)]
            _check(lib.fcm_mlhp_sizes(h, *[C.byref(v) for v in n]))
            M, L, nle, npe = (v.value for v in n)
            IP, LL = C.POINTER(C.c_int), C.POINTER(C.c_longlong)
            self.level = np.empty(M, dtype=np.int32)
            self.t = np.empty((M, 3), dtype=np.int32)
            self.q = np.empty((M, 3), dtype=np.int32)
            _check(lib.fcm_mlhp_functions(h, self.level.ctypes.data_as(IP),
                                          self.t.ctypes.data_as(IP), self.q.ctypes.data_as(IP)))
            self.leaf_level = np.empty(L, dtype=np.int32)
            self.leaf_index = np.empty((L, 3), dtype=np.int32)
            self.leaf_offsets = np.empty(L + 1, dtype=np.int64)
            self.leaf_functions = np.empty(nle, dtype=np.int64)
            _check(lib.fcm_mlhp_leaves(h, self.leaf_level.ctypes.data_as(IP),
                                       self.leaf_index.ctypes.data_as(IP),
                                       self.leaf_offsets.ctypes.data_as(LL),
                                       self.leaf_functions.ctypes.data_as(LL)))
            nodes = 1
            for a in range(prob["dim"]):
                nodes *= prob["cells"][a] + 1
            self.patch_offsets = np.empty(nodes + 1, dtype=np.int64)
            self.patch_functions = np.empty(npe, dtype=np.int64)
            _check(lib.fcm_mlhp_patches(h, self.patch_offsets.ctypes.data_as(LL),
                                        self.patch_functions.ctypes.data_as(LL)))
            self.leaf_classes = np.empty(L, dtype=np.int8)
            _check(lib.fcm_mlhp_leaf_classes(h, self.leaf_classes.ctypes.data_as(
                C.POINTER(C.c_byte))))
            nl = C.c_int()
            self.coarsest = np.empty(M, dtype=np.int32)
            _check(lib.fcm_mlhp_levels(h, C.byref(nl), self.coarsest.ctypes.data_as(IP)))
            self.n_levels = nl.value
        finally:
            lib.fcm_mlhp_destroy(h)
        self.n_functions = M
        self.n_leaves = L


class MlhpOperator:
    """Operator and load of an overlay mesh on the device (fcm_mlhp_op_*):
    leaf matrices integrated and mapped to the leaves' functions on the GPU;
    apply(x) = A x for a CUDA float64 tensor of ndofs entries (field-major,
    the function order of Overlay)."""

    def __init__(self, prob: dict):
        import torch
        self._torch = torch
        g, gm, ph, self._opts, self._keep = descriptors(prob)
        lib = load()
        m = C.c_void_p()
        _check(lib.fcm_mlhp_create(C.byref(g), C.byref(gm), C.byref(m)))
        try:
            self.h = C.c_void_p()
            stream = torch.cuda.current_stream().cuda_stream
            _check(lib.fcm_mlhp_op_create(m, C.byref(g), C.byref(gm), C.byref(ph),
                                          C.c_void_p(stream), C.byref(self.h)))
        finally:
            lib.fcm_mlhp_destroy(m)
        n = C.c_longlong()
        _check(lib.fcm_mlhp_op_ndofs(self.h, C.byref(n)))
        self.ndofs = n.value

    def _empty(self):
        return self._torch.empty(self.ndofs, dtype=self._torch.float64, device="cuda")

    def apply(self, x):
        y = self._empty()
        _check(load().fcm_mlhp_op_apply(self.h, _ptr(x), _ptr(y)))
        return y

    def rhs(self):
        b = self._empty()
        _check(load().fcm_mlhp_op_rhs(self.h, _ptr(b)))
        return b

    def prepare(self):
        """Build the hp-multigrid (fcm_mlhp_op_prepare) with the problem's
        smoother options; returns the number of levels."""
        _check(load().fcm_mlhp_op_prepare(self.h, C.byref(self._opts)))
        self.levels = []
        l = 0
        while True:
            nd, om = C.c_longlong(), C.c_double()
            nb, mb = C.c_int(), C.c_int()
            st = load().fcm_mlhp_op_level(self.h, l, C.byref(nd), C.byref(om), C.byref(nb),
                                          C.byref(mb))
            if st != FCM_OK:
                break
            self.levels.append({"ndofs": nd.value, "omega": om.value, "n_blocks": nb.value,
                                "max_block": mb.value})
            l += 1
        return len(self.levels)

    def vcycle(self, r):
        z = self._empty()
        _check(load().fcm_mlhp_op_vcycle(self.h, _ptr(r), _ptr(z)))
        return z

    def pcg(self, b=None, rtol=1e-8, maxit=500, allow_fail=False):
        x = self._empty()
        inf = fcm_info()
        st = load().fcm_mlhp_op_pcg(self.h, _ptr(b) if b is not None else None, _ptr(x), rtol,
                                    maxit, C.byref(inf))
        _check(st, allow=(FCM_E_NOT_CONVERGED, FCM_E_BREAKDOWN) if allow_fail else ())
        d = inf.as_dict()
        d["status"] = st
        return x, d

    def close(self):
        if self.h:
            load().fcm_mlhp_op_destroy(self.h)
            self.h = None


def measure_fma_peak(prec: int) -> float:
    """FMA throughput of the current GPU in TFLOP/s (FCM_FP64 or FCM_MIXED = FP32)."""
    t = C.c_double()
    _check(load().fcm_measure_fma_peak(prec, C.byref(t)))
    return t.value


def restriction_1d(p: int, dk: int, pos: int) -> np.ndarray:
    """S[i, j]: coefficient of sub-interval mode i in ancestor mode j, for
    sub-interval pos of 2^dk (fcm_mlhp_restriction_1d)."""
    out = np.empty((p + 1) * (p + 1), dtype=np.float64)
    _check(load().fcm_mlhp_restriction_1d(p, dk, pos, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out.reshape(p + 1, p + 1)


def descriptors(prob: dict, build_mixed: bool = True):
    """C descriptors for a problem dict of ``fcm_inputs``.  Raises
    ValueError for problem features the library has no descriptor for
    (trunk-space elements, removal of fictitious cells, geometry kinds or
    smoothers it does not know) instead of dropping them."""
    if prob.get("space", "tensor") not in ("tensor", "trunk"):
        raise ValueError("the library discretises with tensor-product or trunk elements")
    if prob.get("drop_outside") and prob.get("space", "tensor") != "trunk":
        raise ValueError("the library removes fictitious cells with trunk elements only")
    if prob["geometry"]["kind"] not in GEOM:
        raise ValueError(f"geometry kind {prob['geometry']['kind']!r} has no library descriptor")
    if prob.get("smoother", "elementwise") not in SMOOTHER:
        raise ValueError(f"smoother {prob['smoother']!r} has no library descriptor")
    d = prob["dim"]
    g = fcm_grid()
    g.dim = d
    for a in range(3):
        g.cells[a] = prob["cells"][a] if a < d else 1
        g.lo[a] = prob["lo"][a] if a < d else 0.0
        g.hi[a] = prob["hi"][a] if a < d else 0.0
    g.p = prob["p"]
    g.overlay_levels = prob.get("overlay_levels", 0)
    g.space = SPACE_TRUNK if prob.get("space", "tensor") == "trunk" else SPACE_TENSOR
    g.drop_outside = 1 if prob.get("drop_outside") else 0
    geo = prob["geometry"]
    kind = geo["kind"]
    if kind == "ball":
        params = list(geo["center"]) + [geo["radius"]]
    elif kind == "voids":
        params = [v for ball in geo["balls"] for v in ball]
    elif kind == "ellipsoid":
        params = list(geo["center"]) + list(geo["axes"]) + [v for row in geo["rot"] for v in row]
    elif kind == "popcorn":
        params = [geo["r0"], geo["A"], geo["sigma"]] + [v for c in geo["centers"] for v in c]
    else:
        params = []
    arr = (C.c_double * max(1, len(params)))(*params)
    gm = fcm_geometry(GEOM[kind], len(params), arr, 1 if geo.get("complement") else 0)
    ph = fcm_physics()
    ph.pde = PDE[prob["pde"]]
    ph.kappa = prob["kappa"]
    ph.E = prob["E"]
    ph.nu = prob["nu"]
    ph.alpha = prob["alpha"]
    ph.beta = prob["beta"]
    src = prob["source"]
    ph.source = SRC[src["kind"]]
    ph.f0 = src.get("f0", 0.0)
    ph.src_a = src.get("a", 0.0)
    dr = prob["dirichlet"]
    ph.dirichlet = DIR[dr["kind"]]
    ph.g = GVAL[dr.get("g", "zero")]
    mask = 0
    for f in dr.get("faces", []):
        mask |= 1 << f
    ph.dirichlet_faces = mask
    tr = prob.get("traction")
    ph.traction_face = tr["face"] if tr else -1
    if tr:
        for a in range(3):
            ph.traction[a] = tr["t"][a] if a < len(tr["t"]) else 0.0
    ph.quad_depth = prob["quad_depth"]
    quads = {"points": QUAD_POINTS, "sumfact": QUAD_SUMFACT}
    if prob.get("quadrature", "points") not in quads:
        raise ValueError(f"quadrature {prob['quadrature']!r}: one of {sorted(quads)}")
    ph.quadrature = quads[prob.get("quadrature", "points")]
    op = fcm_solver_opts()
    op.smoother = SMOOTHER[prob.get("smoother", "elementwise")]
    op.omega = prob["omega"] if prob.get("omega") else 0.0
    op.n_pre = prob["n_pre"]
    op.n_post = prob["n_post"]
    op.coarse_cells = prob["coarse_cells"]
    op.build_mixed = 1 if build_mixed else 0
    return g, gm, ph, op, arr


def _ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Solver:
    """One FCM problem set up on the current CUDA device (fcm_setup)."""

    def __init__(self, prob: dict, build_mixed: bool = True, stream=None):
        import torch
        lib = load()
        self.prob = prob
        g, gm, ph, op, self._keep = descriptors(prob, build_mixed)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = C.c_void_p()
        _check(lib.fcm_setup(C.byref(g), C.byref(gm), C.byref(ph), C.byref(op),
                             C.c_void_p(s.cuda_stream), C.byref(h)))
        self.h = h
        n = C.c_longlong()
        _check(lib.fcm_ndofs(h, C.byref(n)))
        self.ndofs = n.value

    def close(self):
        if getattr(self, "h", None):
            load().fcm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, n=None):
        import torch
        return torch.empty(self.ndofs if n is None else n, dtype=torch.float64, device="cuda")

    def rhs(self):
        b = self._empty()
        _check(load().fcm_rhs(self.h, _ptr(b)))
        return b

    def apply(self, x, prec=FCM_FP64):
        y = self._empty()
        _check(load().fcm_apply(self.h, _ptr(x), _ptr(y), prec))
        return y

    def vcycle(self, r, prec=FCM_FP64):
        z = self._empty()
        _check(load().fcm_vcycle(self.h, _ptr(r), _ptr(z), prec))
        return z

    def num_levels(self):
        n = C.c_int()
        _check(load().fcm_num_levels(self.h, C.byref(n)))
        return n.value

    def level_info(self, level):
        inf = fcm_level_info()
        _check(load().fcm_level_info_get(self.h, level, C.byref(inf)))
        return inf.as_dict()

    def level_op(self, level, op, x, out_size):
        y = self._empty(out_size)
        _check(load().fcm_level_op(self.h, level, op, _ptr(x), _ptr(y)))
        return y

    def cell_classes(self):
        n = int(np.prod(self.prob["cells"]))
        out = np.empty(n, dtype=np.int8)
        _check(load().fcm_cell_classes(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def pcg(self, b=None, rtol=1e-8, maxit=500, prec=FCM_FP64, x=None, allow_fail=False):
        x = self._empty() if x is None else x
        inf = fcm_info()
        st = load().fcm_pcg_solve(self.h, _ptr(b) if b is not None else None, _ptr(x),
                                  rtol, maxit, prec, C.byref(inf))
        _check(st, allow=(FCM_E_NOT_CONVERGED, FCM_E_BREAKDOWN) if allow_fail else ())
        d = inf.as_dict()
        d["status"] = st
        return x, d

    def solve(self, method, b=None, rtol=1e-8, maxit=500, prec=FCM_FP64, x=None,
              allow_fail=False):
        """fcm_solve: METHOD_CG_MG, METHOD_MG (stand-alone multigrid; info["rho"]
        holds the contraction numbers) or METHOD_CG_AS (one-level Schwarz CG)."""
        x = self._empty() if x is None else x
        inf = fcm_info()
        rho = np.zeros(max(1, maxit))
        st = load().fcm_solve(self.h, method, _ptr(b) if b is not None else None, _ptr(x), rtol,
                              maxit, prec, C.byref(inf), rho.ctypes.data_as(C.c_void_p))
        _check(st, allow=(FCM_E_NOT_CONVERGED, FCM_E_BREAKDOWN) if allow_fail else ())
        d = inf.as_dict()
        d["status"] = st
        if method == METHOD_MG:
            d["rho"] = rho[: d["iters"]].copy()
        return x, d

    def profile_op(self, level, which, prec=FCM_FP64, reps=20):
        ms = C.c_double()
        _check(load().fcm_profile_op(self.h, level, which, prec, reps, C.byref(ms)))
        return ms.value

    def op_bytes(self, level, which, prec=FCM_FP64):
        b = C.c_longlong()
        _check(load().fcm_op_bytes(self.h, level, which, prec, C.byref(b)))
        return b.value

    def pcg_host(self, b=None, rtol=1e-8, maxit=500, prec=FCM_FP64, x_host=None):
        """Solve through host buffers (numpy float64)."""
        x = np.empty(self.ndofs) if x_host is None else x_host
        bp = None
        if b is not None:
            b = np.ascontiguousarray(b, dtype=np.float64)
            bp = b.ctypes.data_as(C.c_void_p)
        inf = fcm_info()
        _check(load().fcm_pcg_solve_host(self.h, bp, x.ctypes.data_as(C.c_void_p), rtol, maxit,
                                         prec, C.byref(inf)))
        return x, inf.as_dict()


class Batch:
    """Independent problems set up and solved together (fcm_setup_batch)."""

    def __init__(self, probs, build_mixed: bool = True, threads: int = 0, stream=None):
        import torch
        lib = load()
        n = len(probs)
        self.probs = probs
        descs = [descriptors(p, build_mixed) for p in probs]
        self._keep = [d[4] for d in descs]
        G = (fcm_grid * n)(*[d[0] for d in descs])
        GM = (fcm_geometry * n)(*[d[1] for d in descs])
        PH = (fcm_physics * n)(*[d[2] for d in descs])
        OP = (fcm_solver_opts * n)(*[d[3] for d in descs])
        s = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib.fcm_setup_batch(n, G, GM, PH, OP, threads, C.c_void_p(s.cuda_stream),
                                   C.byref(h)))
        self.h = h
        self.threads = threads
        self.ndofs = []
        for i in range(n):
            hi = C.c_void_p()
            _check(lib.fcm_batch_handle(h, i, C.byref(hi)))
            nd = C.c_longlong()
            _check(lib.fcm_ndofs(hi, C.byref(nd)))
            self.ndofs.append(nd.value)

    def close(self):
        if getattr(self, "h", None):
            load().fcm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pcg(self, xs=None, rtol=1e-8, maxit=500, prec=FCM_FP64, threads=None):
        """threads 0: all instances in lockstep from this thread; -1: the same
        with one graph launch per CG phase; > 0: a pool of that many host
        workers (default: the set-up's thread count)."""
        import torch
        n = len(self.ndofs)
        if xs is None:
            xs = [torch.empty(nd, dtype=torch.float64, device="cuda") for nd in self.ndofs]
        ptrs = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        infos = (fcm_info * n)()
        t = self.threads if threads is None else threads
        _check(load().fcm_pcg_solve_batch(self.h, ptrs, rtol, maxit, prec, t, infos))
        return xs, [i.as_dict() for i in infos]
