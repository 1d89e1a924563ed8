"""Pipelined host I/O (gks2l_run_items): a queue of independent states, each
set from host arrays, advanced and read back, with the copies of
neighbouring items overlapping the computation. Each item's result must be
bit for bit the result of gks2l_set_state, gks2l_advance and
gks2l_get_state on that item alone."""
import numpy as np
import pytest

from paper_2306_04467_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2306_04467_gb300 import gks2l as g  # noqa: E402


def item_states(prob, n):
    """n seeded perturbations of the problem's initial state."""
    rng = np.random.default_rng(41)
    out = []
    for k in range(n):
        a = np.array(prob.avg, dtype=np.float64, copy=True)
        gr = np.array(prob.grad, dtype=np.float64, copy=True)
        a[3] += 0.002 * k * rng.standard_normal(a.shape[1])
        a[1] += 0.001 * k * rng.standard_normal(a.shape[1])
        out.append((np.ascontiguousarray(a), np.ascontiguousarray(gr)))
    return out


def one_by_one(prob, precision, states, n_stages):
    s = g.problem_solver(prob, precision=precision)
    res = []
    for a, gr in states:
        s.set_state(a, gr)
        s.advance(n_stages)
        res.append(s.get_state())
    return res


@pytest.mark.parametrize("precision", [g.GKS2L_FP64, g.GKS2L_FP32])
def test_items_equal_one_by_one(precision):
    """Five items (both staging buffers reused, an odd stage count) from
    numpy arrays, each against its own set/advance/get."""
    prob = inputs.interface_dambreak(24)
    states = item_states(prob, 5)
    ref = one_by_one(prob, precision, states, 5)
    s = g.problem_solver(prob, precision=precision)
    outs = [(np.zeros((6, prob.mesh.n_tri)), np.zeros((6, 2, prob.mesh.n_tri))) for _ in states]
    s.run_items(states, outs, 5)
    for (a, gr), (ra, rg) in zip(outs, ref):
        assert np.array_equal(a, ra) and np.array_equal(gr, rg)
    assert s.stats()["status"] == 0


def test_pinned_tensors_and_a_shared_output():
    """Pinned torch inputs, one output buffer for every item (the last item's
    result remains) and items without gradients (zero gradients in, none
    out)."""
    prob = inputs.interface_dambreak(20)
    states = item_states(prob, 3)
    nt = prob.mesh.n_tri
    pin = [(torch.from_numpy(a.ravel().copy()).pin_memory(), torch.from_numpy(gr.ravel().copy()).pin_memory())
           for a, gr in states]
    oa = torch.zeros(6 * nt, dtype=torch.float64).pin_memory()
    og = torch.zeros(12 * nt, dtype=torch.float64).pin_memory()
    s = g.problem_solver(prob, precision=g.GKS2L_FP32)
    s.run_items(pin, [(oa, og)] * 3, 4)
    ref = one_by_one(prob, g.GKS2L_FP32, states, 4)
    assert np.array_equal(oa.numpy().reshape(6, nt), ref[-1][0])
    assert np.array_equal(og.numpy().reshape(6, 2, nt), ref[-1][1])
    # no gradients: the states start with zero gradients, only averages return
    s.run_items([(states[0][0], None)], [(np.zeros((6, nt)), None)], 2)
    r = g.problem_solver(prob, precision=g.GKS2L_FP32)
    r.set_state(states[0][0])
    r.advance(2)
    assert np.array_equal(s.get_state()[0], r.get_state()[0])


def test_run_items_rejects_bad_arguments():
    prob = inputs.smooth_periodic(4)
    s = g.problem_solver(prob, precision=g.GKS2L_FP32)
    nt = prob.mesh.n_tri
    with pytest.raises(g.GKSError) as e:
        s.run_items([(np.ascontiguousarray(prob.avg), None)], [(None, None)], 2)
    assert e.value.code == g.GKS2L_EINVAL
    with pytest.raises(g.GKSError) as e:
        s.run_items([(np.ascontiguousarray(prob.avg), None)], [(np.zeros((6, nt)), None)], -1)
    assert e.value.code == g.GKS2L_EINVAL
    s.run_items([], [], 2)   # nothing to do
    on_gpu = torch.zeros(6 * nt, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        s.run_items([(on_gpu, None)], [(np.zeros((6, nt)), None)], 2)
