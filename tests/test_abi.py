"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/fcm.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fcm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fcm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fcm_setup", "fcm_vcycle", "fcm_pcg_solve", "fcm_apply", "fcm_destroy",
              "fcm_last_error", "fcm_pcg_solve_host"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2010_00881_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_2010_00881_gb300 import fcm
    assert sorted(fcm.EXPORTS) == declared_functions()


def test_last_error_without_gpu():
    from paper_2010_00881_gb300 import fcm
    lib = fcm.load()
    assert lib.fcm_ndofs(None, None) == fcm.FCM_E_INVALID
    assert b"null" in lib.fcm_last_error()


def test_descriptor_marshalling_roundtrip():
    import fcm_inputs as fi
    from paper_2010_00881_gb300 import fcm
    prob = fi.poisson3d_sphere(cells=32, p=3)
    g, gm, ph, op, keep = fcm.descriptors(prob)
    assert (g.dim, tuple(g.cells), g.p) == (3, (32, 32, 32), 3)
    assert gm.kind == fcm.GEOM["ball"] and gm.n_params == 4
    assert [gm.params[i] for i in range(4)] == [0.5, 0.5, 0.5, 0.45]
    assert ph.alpha == 1e-8 and ph.beta == 1e4 and ph.dirichlet == fcm.DIR["levelset"]
    assert (op.n_pre, op.n_post, op.coarse_cells) == (5, 5, 4)
    prob = fi.square_mms(cells=8, p=2)
    g, gm, ph, op, keep = fcm.descriptors(prob)
    assert ph.dirichlet_faces == 0b1111 and ph.kappa == 10.0
