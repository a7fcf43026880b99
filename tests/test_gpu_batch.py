"""Batched mode (independent FCM instances of uneven grid size, degree and
geometry solved together): every instance must give exactly the result of
solving it alone (the kernels are deterministic), converge to the
tolerance, and take the oracle's iteration count +-1."""
import numpy as np
import pytest

import fcm_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2010_00881_gb300 import FCM_FP64, FCM_MIXED  # noqa: E402
from paper_2010_00881_gb300 import fcm as F  # noqa: E402


def small_batch(n=5):
    out = []
    for i in range(n):
        prob = fi.batch_instance(i)
        c = 4 + (i % 4)          # 4..7 cells per axis: ragged h-levels
        prob["cells"] = (c, c, c)
        prob["p"] = 2 + (i % 2)
        out.append(prob)
    return out


@pytest.fixture(scope="module")
def batch():
    probs = small_batch()
    b = F.Batch(probs, threads=3)
    yield probs, b
    b.close()


@pytest.mark.parametrize("threads", [0, -1, 3])
@pytest.mark.parametrize("prec", [FCM_FP64, FCM_MIXED])
def test_batch_equals_individual_solves(batch, prec, threads):
    """threads 0: all instances in lockstep from one host thread; -1: the
    same with one graph launch per CG phase; 3: a pool of host workers.
    All run each instance's work exactly as alone."""
    probs, b = batch
    xs, infos = b.pcg(rtol=1e-8, prec=prec, threads=threads)
    for prob, x, info in zip(probs, xs, infos):
        s = F.Solver(prob)
        xi, ii = s.pcg(rtol=1e-8, prec=prec)
        assert info["iters"] == ii["iters"]
        assert info["relres_true"] <= 1e-8
        assert torch.equal(x, xi)
        s.close()


def _oracle_batch_problems():
    out = []
    for i, p in enumerate((2, 3, 4, 2)):
        prob = fi.batch_instance(10 + i)
        c = 5 + (i % 2)
        prob["cells"] = (c, c, c)
        prob["p"] = p
        out.append(prob)
    return out


@pytest.fixture(scope="module")
def oracle_batch():
    """Four instances of the batch workload (rotated ellipsoids, p = 2..4,
    5 or 6 cells per axis) with their oracle hierarchies and solutions."""
    from oracle import multigrid as mg
    probs = _oracle_batch_problems()
    Hs = [mg.Hierarchy(prob) for prob in probs]
    sols = [mg.pcg(H.A, H.b, H.vcycle, rtol=1e-8) for H in Hs]
    b = F.Batch(probs, threads=2)
    yield probs, Hs, sols, b
    b.close()


@pytest.mark.parametrize("prec", [FCM_FP64, FCM_MIXED])
def test_batch_matches_oracle(oracle_batch, prec):
    """Every instance of a batched solve takes the oracle's iteration count
    +-1 and meets the tolerance in the oracle's own residual b - A x."""
    import scipy.sparse.linalg as spla
    probs, Hs, sols, b = oracle_batch
    xs, infos = b.pcg(rtol=1e-8, prec=prec, threads=0)
    for i, (H, (xo, ko, _), x, info) in enumerate(zip(Hs, sols, xs, infos)):
        x = x.cpu().numpy()
        assert abs(info["iters"] - ko) <= 1, (i, prec, info["iters"], ko)
        assert np.linalg.norm(H.b - H.A @ x) / np.linalg.norm(H.b) <= 1.01e-8, i
        # two Krylov paths to residual 1e-8: ||x - xo||_A is bounded by the
        # residuals' A^-1 norms (slack 1.5)
        lu = spla.splu(H.A.tocsc())

        def rnorm_ainv(v):
            r = H.b - H.A @ v
            return np.sqrt(abs(r @ lu.solve(r)))

        e = x - xo
        ea = np.sqrt(max(e @ (H.A @ e), 0.0))
        assert ea <= 1.5 * (rnorm_ainv(x) + rnorm_ainv(xo)) + 1e-300, (i, prec)


def test_batch_reports_failing_instance():
    probs = small_batch(3)
    probs[2] = dict(probs[2], p=0)
    with pytest.raises(F.FcmError) as e:
        F.Batch(probs, threads=2)
    assert e.value.status == F.FCM_E_INVALID
    assert "instance 2" in str(e.value)
