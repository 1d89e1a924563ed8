"""The allocation-free CFL/mass entry point agrees with the bound library.

gks2l_cfl_mass_noalloc serves callers that cannot call cudaMalloc -- code
inside another framework's memory pool, a process whose device memory is all
reserved up front, a loop that must not allocate -- and so cannot give the
library its workspace; it keeps its scratch in a fixed device array. Here it
is called through the C ABI on two states in a row and checked against what a
bound context reports for the same states: the layer masses gks2l_stats gives
for the state, and the step size gks2l_stats gives for the step taken from
that state. A second mesh is large enough that the entry point caps its grid
and strides over the cells. This file is collected last on purpose.
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


@pytest.mark.parametrize("case", ["smooth_24sq", "lake_512sq"])
def test_noalloc_matches_bound_context_on_two_calls(case):
    """1,152 triangles (5 blocks), and 524,288 triangles: more than the 1024
    blocks x 256 threads of one pass, so the grid is capped and each thread
    strides over several cells."""
    prob = inputs.smooth_periodic(24) if case == "smooth_24sq" else inputs.lake_at_rest(512)
    if case == "lake_512sq":
        assert prob.mesh.n_tri > 1024 * 256
    s = g.problem_solver(prob, precision=g.GKS2L_FP64)
    dev = torch.device("cuda")
    area, dX = cell_geometry(prob.mesh)
    area_t = torch.tensor(area, dtype=torch.float64, device=dev)
    dX_t = torch.tensor(dX, dtype=torch.float64, device=dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    state = torch.tensor(np.ascontiguousarray(prob.avg).ravel(), dtype=torch.float64, device=dev)
    for call in range(2):
        before = s.stats()               # masses of the current state
        g.cfl_mass_noalloc(state, area_t, dX_t, prob.g, prob.cfl, out)
        torch.cuda.synchronize()
        dt, m1, m2, bad = out.tolist()
        s.advance(2)                     # one step from that state
        after = s.stats()                # its step size
        assert after["status"] == 0 and bad == 0
        np.testing.assert_allclose(dt, after["dt"], rtol=1e-13)
        np.testing.assert_allclose([m1, m2], before["mass"], rtol=1e-12)
        s.get_state_device(state)        # next call: the state after the step
        torch.cuda.synchronize()


def test_noalloc_counts_unusable_cells():
    """A NaN depth, a negative depth and a zero depth are counted and left
    out of the step; the remaining cells give the bound context's step."""
    prob = inputs.smooth_periodic(24)
    dev = torch.device("cuda")
    area, dX = cell_geometry(prob.mesh)
    avg = np.ascontiguousarray(prob.avg).copy()
    good = avg.copy()
    avg[3, 7], avg[0, 100], avg[3, 500] = np.nan, -0.2, 0.0
    out = torch.empty(4, dtype=torch.float64, device=dev)
    args = [torch.tensor(x, dtype=torch.float64, device=dev) for x in (avg.ravel(), area, dX)]
    g.cfl_mass_noalloc(*args, prob.g, prob.cfl, out)
    torch.cuda.synchronize()
    dt, _, _, bad = out.tolist()
    assert bad == 3
    keep = np.ones(prob.mesh.n_tri, bool)
    keep[[7, 100, 500]] = False
    um = np.maximum(*[np.hypot(good[b + 1], good[b + 2]) / good[b] + np.sqrt(prob.g * good[b]) for b in (0, 3)])
    np.testing.assert_allclose(dt, prob.cfl * (dX / um)[keep].min(), rtol=1e-13)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    dev = torch.device("cuda")
    buf = torch.zeros(6, dtype=torch.float64, device=dev)
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    L = g.load()
    rc = L.gks2l_cfl_mass_noalloc((1 << 28) + 1, g._P(buf.data_ptr()), g._P(buf.data_ptr()),
                                  g._P(buf.data_ptr()), 9.81, 0.5, g._P(out.data_ptr()), None)
    assert rc == g.GKS2L_ETOOBIG and L.gks2l_error_string(rc).startswith(b"size beyond")
