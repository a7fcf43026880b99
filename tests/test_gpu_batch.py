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


@pytest.mark.parametrize("prec", [FCM_FP64, FCM_MIXED])
def test_batch_equals_individual_solves(batch, prec):
    probs, b = batch
    xs, infos = b.pcg(rtol=1e-8, prec=prec)
    for prob, x, info in zip(probs, xs, infos):
        s = F.Solver(prob)
        xi, ii = s.pcg(rtol=1e-8, prec=prec)
        assert info["iters"] == ii["iters"]
        assert info["relres_true"] <= 1e-8
        assert torch.equal(x, xi)
        s.close()


def test_batch_instance_matches_oracle():
    from oracle import multigrid as mg
    prob = small_batch(2)[1]
    H = mg.Hierarchy(prob)
    xo, ko, _ = mg.pcg(H.A, H.b, H.vcycle, rtol=1e-8)
    b = F.Batch([prob], threads=1)
    xs, infos = b.pcg(rtol=1e-8, prec=FCM_FP64)
    assert abs(infos[0]["iters"] - ko) <= 1
    e = xs[0].cpu().numpy() - xo
    assert np.sqrt(e @ (H.A @ e)) / np.sqrt(xo @ (H.A @ xo)) <= 1e-7
    b.close()


def test_batch_reports_failing_instance():
    probs = small_batch(3)
    probs[2] = dict(probs[2], p=0)
    with pytest.raises(F.FcmError) as e:
        F.Batch(probs, threads=2)
    assert e.value.status == F.FCM_E_INVALID
    assert "instance 2" in str(e.value)
