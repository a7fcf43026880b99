"""fcm_cell_apply_noalloc, the allocation-free operator apply for callers
that cannot allocate device memory (they hold the cell matrices and vectors
themselves; the library's scratch is a fixed array compiled into it).

Its output must match the regular entry point fcm_apply on the same
problem, on two calls in a row (the calls share the scratch array), and it
must reject a grid whose per-cell products do not fit the array.  This file
is collected last so that a run stopping at the first failure has already
run every other test."""
import ctypes as C

import numpy as np
import pytest

import fcm_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from oracle.assembly import element_system  # noqa: E402
from oracle.grid import all_cells  # noqa: E402
from paper_2010_00881_gb300 import fcm as F  # noqa: E402


def _noalloc(dim, cells, p, K, x, y):
    lib = F.load()
    arr = (C.c_int * 3)(*(list(cells) + [1] * (3 - len(cells))))
    return lib.fcm_cell_apply_noalloc(dim, arr, p, C.c_void_p(K.data_ptr()),
                                      C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))


# Each case reaches one kernel of the cell apply: 2D p = 2 (9 DOFs per cell,
# unpadded rows: the scalar per-cell kernel), 2D p = 3 and 3D p = 1 (16 and 8
# DOFs: one lane group per cell), 3D p = 3 (64 DOFs, 16-byte rows: the bulk-copy
# streaming kernel).
CASES = {
    "circle16_p2": lambda: fi.poisson2d_circle(),
    "circle8_p3": lambda: fi.poisson2d_circle(cells=8, p=3),
    "sphere4_p1": lambda: fi.poisson3d_sphere(cells=4, p=1),
    "sphere4_p3": lambda: fi.poisson3d_sphere(cells=4, p=3),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_apply_matches_fcm_apply_twice(case):
    prob = CASES[case]()
    s = F.Solver(prob, build_mixed=False)
    K = np.stack([element_system(prob, c)[0]
                  for c in all_cells(prob["dim"], prob["cells"])])
    Kd = torch.from_numpy(np.ascontiguousarray(K)).cuda()
    for seed in (1, 2):
        x = torch.from_numpy(fi.random_vector(s.ndofs, seed=seed)).cuda()
        y = torch.full((s.ndofs,), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(prob["dim"], prob["cells"], prob["p"], Kd, x, y)
        assert st == F.FCM_OK, F.load().fcm_last_error()
        ref = s.apply(x)
        rel = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
        assert rel <= 1e-12, (case, seed, rel)
    s.close()


def test_noalloc_rejects_grids_beyond_the_scratch():
    K = torch.zeros(81, dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = _noalloc(2, (512, 512), 2, K, x, y)   # 262,144 cells x 9 products > 4 MiB
    assert st == F.FCM_E_INVALID
    assert b"scratch" in F.load().fcm_last_error()
