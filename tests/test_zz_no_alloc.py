"""The allocation-free CFL/mass entry point agrees with the bound library.

gks2l_cfl_mass_noalloc serves callers that cannot call cudaMalloc and so
cannot give the library its workspace; it keeps its scratch in a fixed device
array. Here it is called through the C ABI on two states in a row and checked
against what a bound context reports for the same states: the layer masses
gks2l_stats gives for the state, and the step size gks2l_stats gives for the
step taken from that state. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2306_04467_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2306_04467_gb300 import gks2l as g  # noqa: E402


def cell_geometry(mesh):
    P = mesh.xy[mesh.tri]
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                        (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    per = sum(np.hypot(*(P[:, (k + 1) % 3] - P[:, k]).T) for k in range(3))
    return area, 4.0 * area / per


def test_noalloc_matches_bound_context_on_two_calls():
    prob = inputs.smooth_periodic(24)
    s = g.problem_solver(prob, precision=g.GKS2L_FP64)
    dev = torch.device("cuda")
    area, dX = cell_geometry(prob.mesh)
    area_t = torch.tensor(area, dtype=torch.float64, device=dev)
    dX_t = torch.tensor(dX, dtype=torch.float64, device=dev)
    out = torch.empty(3, dtype=torch.float64, device=dev)
    state = torch.tensor(np.ascontiguousarray(prob.avg).ravel(), dtype=torch.float64, device=dev)
    for call in range(2):
        before = s.stats()               # masses of the current state
        g.cfl_mass_noalloc(state, area_t, dX_t, prob.g, prob.cfl, out)
        torch.cuda.synchronize()
        dt, m1, m2 = out.tolist()
        s.advance(2)                     # one step from that state
        after = s.stats()                # its step size
        assert after["status"] == 0
        np.testing.assert_allclose(dt, after["dt"], rtol=1e-13)
        np.testing.assert_allclose([m1, m2], before["mass"], rtol=1e-13)
        s.get_state_device(state)        # next call: the state after the step
        torch.cuda.synchronize()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    dev = torch.device("cuda")
    buf = torch.zeros(6, dtype=torch.float64, device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    L = g.load()
    rc = L.gks2l_cfl_mass_noalloc((1 << 28) + 1, g._P(buf.data_ptr()), g._P(buf.data_ptr()),
                                  g._P(buf.data_ptr()), 9.81, 0.5, g._P(out.data_ptr()), None)
    assert rc == -9 and L.gks2l_error_string(rc).startswith(b"size beyond")
