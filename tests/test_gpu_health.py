"""Health statuses raised by host-made faults (no GPU fault, trap or hang):
a non-finite or non-positive depth handed to gks2l_set_state, and a
reconstruction whose operator staging is told to give up after one poll.
Each call reports its GKS2L_E* code, and the context (or, for the staging
case, the CUDA context) stays usable: a good state set afterwards advances
exactly like a fresh run."""
import numpy as np
import pytest

from paper_2306_04467_gb300 import gks2l as g
from paper_2306_04467_gb300 import inputs

pytestmark = pytest.mark.gpu

FORMS = [g.GKS2L_FP64, g.GKS2L_FP32]


def _fresh(prob, precision, stages):
    s = g.problem_solver(prob, precision=precision)
    s.advance(stages)
    return s.get_state()


@pytest.mark.parametrize("precision", FORMS)
def test_nan_depth_is_reported_and_the_context_recovers(precision):
    prob = inputs.smooth_periodic(16)
    s = g.problem_solver(prob, precision=precision)
    bad = prob.avg.copy()
    bad[3, 17] = np.nan
    s.set_state(bad, prob.grad)
    assert s.stats()["status"] == g.GKS2L_ENONFINITE
    with pytest.raises(g.GKSError) as e:
        s.advance(2)
    assert e.value.code == g.GKS2L_ENONFINITE
    s.set_state(prob.avg, prob.grad)
    assert s.stats()["status"] == 0
    s.advance(6)
    a, gr = s.get_state()
    a0, g0 = _fresh(prob, precision, 6)
    assert np.array_equal(a, a0) and np.array_equal(gr, g0)


@pytest.mark.parametrize("precision", FORMS)
def test_negative_depth_is_reported_and_the_context_recovers(precision):
    prob = inputs.smooth_periodic(16)
    s = g.problem_solver(prob, precision=precision)
    bad = prob.avg.copy()
    bad[0, 5] = -0.1      # the upper layer's depth in one cell
    s.set_state(bad, prob.grad)
    assert s.stats()["status"] == g.GKS2L_ENEGDEPTH
    s.set_state(prob.avg, prob.grad)
    assert s.stats()["status"] == 0
    s.advance(4)
    a, _ = s.get_state()
    a0, _ = _fresh(prob, precision, 4)
    assert np.array_equal(a, a0)


@pytest.mark.parametrize("precision", FORMS)
def test_staging_that_gives_up_reports_timeout(precision):
    """staging_poll_limit = 1: each reconstruction block gives up on its
    operator copy without polling, records the timeout, waits for the copy
    (up to a second) and leaves without writing. The stage reports
    GKS2L_ETIMEOUT; a context with the default wait on the same device then
    runs exactly like any fresh one."""
    prob = inputs.lake_at_rest(64)
    s = g.problem_solver(prob, precision=precision, staging_poll_limit=1)
    with pytest.raises(g.GKSError) as e:
        s.advance(2)
    assert e.value.code == g.GKS2L_ETIMEOUT
    assert s.stats()["status"] == g.GKS2L_ETIMEOUT
    s.close()
    a, _ = _fresh(prob, precision, 4)
    b, _ = _fresh(prob, precision, 4)
    assert np.array_equal(a, b) and np.isfinite(a).all()


def test_negative_poll_limit_is_rejected():
    prob = inputs.smooth_periodic(8)
    with pytest.raises(g.GKSError) as e:
        g.problem_solver(prob, staging_poll_limit=-1)
    assert e.value.code == g.GKS2L_EINVAL
