"""Batched ensembles and launch shapes, through the C ABI.

An ensemble is many independent problems (each with its own mesh, time step
and clock) advanced together: every kernel of a stage covers all instances'
cells and edges, and one captured CUDA graph runs a whole step. Checked here:
instances advance exactly as they would alone; each conserves its own mass;
the kernels' launch shapes, and the autotuner that picks them, leave every
result unchanged; and the benchmark's ensemble (256 instances of 5k to 200k
triangles) holds its invariants at full size.
"""
import numpy as np
import pytest

from paper_2306_04467_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2306_04467_gb300 import gks2l as g  # noqa: E402

from test_gpu_parity import areas  # noqa: E402


def ensemble(probs, precision):
    par = g.default_params(g=probs[0].g, chi=probs[0].chi, cfl=probs[0].cfl, precision=precision)
    s = g.Solver([p.mesh for p in probs], par, np.concatenate([p.b_vert for p in probs]))
    s.set_state(np.concatenate([p.avg for p in probs], axis=1), np.concatenate([p.grad for p in probs], axis=2))
    return s


@pytest.mark.parametrize("precision", [g.GKS2L_FP64, g.GKS2L_FP32])
def test_launch_shapes_leave_results_unchanged(precision):
    prob = inputs.interface_dambreak(24)
    ref = g.problem_solver(prob, precision=precision)
    ref.advance(20)
    a0, g0 = ref.get_state()
    for shapes in ([0, 0, 0], [2, 2, 2], [3, 3, 3], [4, 4, 4], [0, 3, 2]):
        s = g.problem_solver(prob, precision=precision)
        s.set_launch_shapes(shapes)
        s.advance(20)
        a, gr = s.get_state()
        assert np.array_equal(a, a0) and np.array_equal(gr, g0), shapes


def test_autotune_advances_like_advance():
    prob = inputs.lake_at_rest(48)
    prob.avg[3] += 0.01 * np.sin(np.arange(prob.mesh.n_tri))
    s = g.problem_solver(prob, precision=g.GKS2L_FP32)
    shapes = s.autotune(1)
    assert len(shapes) == 4 and all(0 <= b < 5 for b in shapes[:3]) and shapes[3] == 0
    s.advance(6)
    a, gr = s.get_state()
    ref = g.problem_solver(prob, precision=g.GKS2L_FP32)
    ref.advance(5 * 2 + 6)
    b, h = ref.get_state()
    assert np.array_equal(a, b) and np.array_equal(gr, h)
    with pytest.raises(g.GKSError):
        s.set_launch_shapes([0, 5, 0])


@pytest.mark.parametrize("precision", [g.GKS2L_FP64, g.GKS2L_FP32])
def test_uneven_ensemble_matches_single_runs(precision):
    sizes = inputs.ensemble_sizes(12, lo=300, hi=12000, seed=41)
    probs = [inputs.ensemble_member(int(n), seed=500 + i) for i, n in enumerate(sizes)]
    ens = ensemble(probs, precision)
    t_end = 0.02
    ens.advance(400, t_end=t_end)
    a, gr = ens.get_state()
    assert ens.stats()["status"] == 0
    off = 0
    for i, p in enumerate(probs):
        n = p.mesh.n_tri
        ai, gi = a[:, off:off + n], gr[:, :, off:off + n]
        # every instance lands on t_end with its own time steps and keeps its mass
        area = areas(p.mesh)
        for v in (0, 3):
            m0, m1 = area @ p.avg[v], area @ ai[v]
            assert abs(m1 - m0) <= 1e-12 * m0, (i, v)
        if i % 4 == 0:
            s = g.Solver(p.mesh, g.default_params(g=p.g, chi=p.chi, cfl=p.cfl, precision=precision), p.b_vert)
            s.set_state(p.avg, p.grad)
            t = s.advance(400, t_end=t_end)
            assert abs(t - t_end) < 1e-12
            b, h = s.get_state()
            assert np.array_equal(ai, b) and np.array_equal(gi, h), i
        off += n


def test_full_size_ensemble_invariants():
    """The benchmark's ensemble: 256 instances, 5k to 200k triangles
    (log-uniform), Fourier bathymetry, FP32. After autotuning and 20 steps,
    each instance conserves both layers' mass and stays finite."""
    sizes = inputs.ensemble_sizes(256)
    probs = [inputs.ensemble_member(int(n), seed=3000 + i) for i, n in enumerate(sizes)]
    n_tri = sum(p.mesh.n_tri for p in probs)
    assert 5.0e6 < n_tri < 3.0e7
    ens = ensemble(probs, g.GKS2L_FP32)
    ens.autotune(1)
    ens.advance(40)
    a, _ = ens.get_state()
    assert ens.stats()["status"] == 0 and np.isfinite(a).all()
    off = 0
    for p in probs:
        n = p.mesh.n_tri
        area = areas(p.mesh)
        for v in (0, 3):
            m0, m1 = area @ p.avg[v], area @ a[v, off:off + n]
            assert abs(m1 - m0) <= 1e-12 * m0
        off += n
