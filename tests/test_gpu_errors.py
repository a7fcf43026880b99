"""Error behaviour of the C ABI on the GPU: invalid descriptors and inputs
return statuses (no fault, no hang), and a solve that runs out of
iterations reports FCM_E_NOT_CONVERGED with its iteration count."""
import ctypes as C
import math

import numpy as np
import pytest

import fcm_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2010_00881_gb300 import fcm as F  # noqa: E402


def _setup(prob, **over):
    lib = F.load()
    g, gm, ph, op, keep = F.descriptors(prob)
    for k, v in over.items():
        obj, field = k.split(".")
        setattr({"g": g, "ph": ph, "op": op, "gm": gm}[obj], field, v)
    h = C.c_void_p()
    st = lib.fcm_setup(C.byref(g), C.byref(gm), C.byref(ph), C.byref(op), None, C.byref(h))
    return st, h


@pytest.mark.parametrize("over,status", [
    ({"g.dim": 4}, F.FCM_E_INVALID),
    ({"g.p": 0}, F.FCM_E_INVALID),
    ({"ph.alpha": 0.0}, F.FCM_E_INVALID),
    ({"ph.alpha": float("nan")}, F.FCM_E_INVALID),
    ({"op.coarse_cells": 0}, F.FCM_E_INVALID),
    ({"g.overlay_levels": 2}, F.FCM_E_UNSUPPORTED),
    ({"op.smoother": 1}, F.FCM_E_UNSUPPORTED),
    ({"ph.quadrature": 7}, F.FCM_E_INVALID),
])
def test_invalid_setup(over, status):
    st, h = _setup(fi.poisson2d_circle(cells=4), **over)
    assert st == status
    assert not h.value
    assert len(F.load().fcm_last_error()) > 0


@pytest.mark.parametrize("prob", [fi.poisson3d_sphere_mlhp(cells=4),
                                  dict(fi.poisson2d_circle(cells=4), smoother="patchwise")])
def test_problem_dicts_beyond_the_gpu_path(prob):
    """Overlay and patchwise problem dicts reach fcm_setup through the
    binding, which rejects them before launching anything."""
    with pytest.raises(F.FcmError) as e:
        F.Solver(prob)
    assert e.value.status == F.FCM_E_UNSUPPORTED


def test_nan_rhs_rejected():
    s = F.Solver(fi.poisson2d_circle(cells=8))
    b = s.rhs()
    b[3] = math.nan
    with pytest.raises(F.FcmError) as e:
        s.pcg(b=b)
    assert e.value.status == F.FCM_E_INVALID
    s.close()


def test_not_converged_reports_iterations():
    s = F.Solver(fi.poisson2d_circle(cells=8))
    x, info = s.pcg(rtol=1e-14, maxit=2, allow_fail=True)
    assert info["status"] == F.FCM_E_NOT_CONVERGED
    assert info["iters"] == 2
    assert info["relres_true"] > 1e-14
    s.close()


def test_null_arguments():
    lib = F.load()
    assert lib.fcm_ndofs(None, None) == F.FCM_E_INVALID
    assert lib.fcm_apply(None, None, None, 0) == F.FCM_E_INVALID
    assert lib.fcm_pcg_solve(None, None, None, 1e-8, 10, 0, None) == F.FCM_E_INVALID
