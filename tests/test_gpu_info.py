"""Solve statistics reported through fcm_info: the algorithmic byte count of
a solve (bytes_moved_est) and the kernel launch count.

Both are sums over the launches a solve makes, so a CG iteration adds the
same amount every time: the increments between solves stopped after k,
k + 1 and k + 2 iterations are equal.  Each iteration runs one V-cycle
(n_pre + n_post smoothing steps on every level >= 1) and one FP64 operator
apply, so its bytes are at least those of the finest level's cell
operations in those steps (fcm_op_bytes).  The set-up phases add up within
the set-up's wall time.
"""
import pytest

import fcm_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2010_00881_gb300 import FCM_FP64, FCM_MIXED, Solver  # noqa: E402


@pytest.fixture(scope="module")
def solver():
    s = Solver(fi.poisson3d_sphere(cells=6, p=3))
    yield s
    s.close()


@pytest.mark.parametrize("prec", [FCM_FP64, FCM_MIXED])
def test_bytes_and_launches_per_iteration_are_constant(solver, prec):
    s = solver
    stats = []
    for k in (3, 4, 5):
        _, info = s.pcg(rtol=1e-300, maxit=k, prec=prec, allow_fail=True)
        assert info["iters"] == k
        stats.append((info["bytes_moved_est"], info["kernel_launches"]))
    (b3, l3), (b4, l4), (b5, l5) = stats
    assert b4 - b3 == b5 - b4 > 0
    assert l4 - l3 == l5 - l4 > 0
    top = s.num_levels() - 1
    smoothing_steps = 10      # n_pre + n_post of the default options
    # cell operations alone: the FP64 operator of the CG, and on the finest
    # level of the V-cycle one smoother per step and one operator per step
    # but the first (the gathers, transfers and coarser levels come on top,
    # less than the finest level's cell operations again on these grids)
    lower = (s.op_bytes(top, 0, FCM_FP64)
             + smoothing_steps * s.op_bytes(top, 1, prec)
             + (smoothing_steps - 1) * s.op_bytes(top, 0, prec))
    assert lower <= b4 - b3 <= 5 * lower, (b4 - b3, lower)


def test_bytes_of_a_converged_solve(solver):
    _, info = solver.pcg(rtol=1e-8, prec=FCM_MIXED)
    assert info["bytes_moved_est"] > 0
    print(f"bytes per solve {info['bytes_moved_est'] / 1e9:.3f} GB, "
          f"{info['bytes_moved_est'] / (info['solve_ms'] * 1e-3) / 1e9:.0f} GB/s (host clock)")


def test_setup_phases_add_up_within_the_setup_time(solver):
    """fcm_info.setup_phase_ms: five non-negative phase durations (CUDA
    events on the handle's stream) that together stay within the wall time
    of fcm_setup, the geometry phase (space-tree integration) non-zero."""
    _, info = solver.pcg(rtol=1e-8)
    ph = info["setup_phase_ms"]
    assert len(ph) == 5 and min(ph) >= 0.0
    assert ph[0] > 0.0
    assert sum(ph) <= info["setup_ms"] * 1.001 + 0.05
