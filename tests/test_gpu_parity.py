"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Relative difference: |gpu - oracle| / scale with one scale per variable, the
largest |oracle| value of that variable, floored for variables that are zero
(discharges at rest) at 1e-3 of the layer's depth times its wave speed, and
for gradients at that scale over the smallest cell size.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2306_04467_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2306_04467_gb300 import gks2l as g  # noqa: E402

FP64 = g.GKS2L_FP64
FP32 = g.GKS2L_FP32


def areas(mesh):
    P = mesh.xy[mesh.tri]
    return 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))


def scales(prob, ao, go):
    hmax = max(np.abs(ao[0]).max(), np.abs(ao[3]).max())
    floor_v = 1e-3 * hmax * math.sqrt(prob.g * hmax)
    hmin = math.sqrt(areas(prob.mesh).min())
    sa = np.maximum(np.abs(ao).max(axis=1), floor_v)
    sg = np.maximum(np.abs(go).max(axis=(1, 2)), floor_v / hmin)
    return sa, sg


def max_rel(prob, a, gr, ao, go):
    sa, sg = scales(prob, ao, go)
    ra = (np.abs(a - ao).max(axis=1) / sa).max()
    rg = (np.abs(gr - go).max(axis=(1, 2)) / sg).max()
    return ra, rg


def run_both(prob, n_stages, t_end=0.0, precision=FP64):
    s = g.problem_solver(prob, precision=precision)
    if t_end > 0:
        # in chunks: gks2l_advance enqueues every stage it is asked for
        done, tg = 0, 0.0
        while done < n_stages and tg < t_end * (1 - 1e-12):
            tg = s.advance(min(200, n_stages - done), t_end=t_end)
            done += 200
    else:
        tg = s.advance(n_stages, t_end=t_end)
    a, gr = s.get_state()
    st = s.stats()
    o = Oracle.from_problem(prob)
    o.advance(n_stages, t_end=t_end)
    ao, go = o.get_state()
    return (a, gr, tg, st), (ao, go, o.t)


def test_fp64_matches_oracle_config1_100_stages():
    prob = inputs.smooth_periodic(16)
    (a, gr, tg, st), (ao, go, to) = run_both(prob, 100)
    assert st["status"] == 0
    assert abs(tg - to) <= 1e-14 * to
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (ra, rg)


def test_fp64_matches_oracle_to_t_end():
    prob = inputs.smooth_periodic(16)
    (a, gr, tg, st), (ao, go, to) = run_both(prob, 10 ** 6, t_end=prob.t_end)
    assert abs(tg - prob.t_end) < 1e-12 and abs(to - prob.t_end) < 1e-12
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (ra, rg)


def test_advance_to_an_end_time_stops_when_every_instance_arrives():
    """One call asking for a million stages with an end time runs only the
    steps needed (checked every 32 steps): no more than 64 stages beyond
    stepping one step at a time, and the same state bit for bit."""
    prob = inputs.smooth_periodic(16)
    s1 = g.problem_solver(prob)
    t1 = s1.advance(10 ** 6, t_end=prob.t_end)
    a1, g1 = s1.get_state()
    s2 = g.problem_solver(prob)
    t2 = 0.0
    while t2 < prob.t_end * (1 - 1e-12):
        t2 = s2.advance(2, t_end=prob.t_end)
    a2, g2 = s2.get_state()
    assert t1 == t2 and abs(t1 - prob.t_end) < 1e-12
    assert s2.stats()["stages"] <= s1.stats()["stages"] <= s2.stats()["stages"] + 64
    assert np.array_equal(a1, a2) and np.array_equal(g1, g2)


@pytest.mark.parametrize("case", ["dambreak", "lake", "translation", "rect_walls", "tiny_periodic", "tiny_walls"])
def test_fp64_matches_oracle_cases(case):
    if case == "dambreak":
        prob, n = inputs.interface_dambreak(16), 60
    elif case == "lake":
        prob, n = inputs.lake_at_rest(20), 30
    elif case == "translation":
        prob, n = inputs.translation(12), 40
    elif case == "rect_walls":
        prob = inputs.lake_at_rest(9, domain=(0.0, 1.7, 0.0, 1.0))
        prob.avg[3] += 0.01 * np.sin(np.arange(prob.mesh.n_tri))  # disturb the interface
        n = 30
    elif case == "tiny_periodic":
        prob, n = inputs.smooth_periodic(4), 20
    else:
        prob = inputs.lake_at_rest(3)
        prob.avg[0] *= 1.0 + 0.05 * np.cos(np.arange(prob.mesh.n_tri))
        n = 20
    (a, gr, tg, st), (ao, go, to) = run_both(prob, n)
    assert st["status"] == 0
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (case, ra, rg)


def test_odd_stage_counts_are_exact():
    prob = inputs.smooth_periodic(16)
    s1 = g.problem_solver(prob)
    s1.advance(3)
    s1.advance(1)
    a1, g1 = s1.get_state()
    s2 = g.problem_solver(prob)
    s2.advance(4)
    a2, g2 = s2.get_state()
    assert np.array_equal(a1, a2) and np.array_equal(g1, g2)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_checkpoint_restart_is_bitwise(precision):
    """A state read out with gks2l_get_state after 50 stages and set into a
    new context continues exactly as the uninterrupted run: 50 + 50 stages
    equal 100 stages bit for bit (the device keeps the state's own gradients,
    and a restarted run takes the CFL step the way the running one does)."""
    prob = inputs.interface_dambreak(24)
    full = g.problem_solver(prob, precision=precision)
    full.advance(100)
    a100, g100 = full.get_state()
    first = g.problem_solver(prob, precision=precision)
    first.advance(50)
    ca, cg = first.get_state()
    second = g.problem_solver(prob, precision=precision)
    second.set_state(ca, cg)
    ra, rg = second.get_state()
    assert np.array_equal(ra, ca) and np.array_equal(rg, cg)    # the round trip itself
    second.advance(50)
    b100, h100 = second.get_state()
    assert np.array_equal(b100, a100) and np.array_equal(h100, g100)
    assert full.stats()["status"] == 0 and second.stats()["status"] == 0


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_lake_at_rest_is_preserved(precision):
    prob = inputs.lake_at_rest(96)
    s = g.problem_solver(prob, precision=precision)
    s.advance(200)
    a, _ = s.get_state()
    bav = prob.b_vert[prob.mesh.tri].mean(1)
    assert np.abs(a[3] + bav - 0.8).max() <= 1e-12
    assert np.abs(a[0] - 0.2).max() <= 1e-12
    assert np.abs(a[[1, 2, 4, 5]]).max() <= 1e-12
    assert s.stats()["status"] == 0


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("case", ["periodic", "walls"])
def test_mass_is_conserved(precision, case):
    prob = inputs.smooth_periodic(48) if case == "periodic" else inputs.interface_dambreak(48)
    area = areas(prob.mesh)
    s = g.problem_solver(prob, precision=precision)
    m0 = np.array([area @ prob.avg[3], area @ prob.avg[0]])
    s.advance(100)
    a, _ = s.get_state()
    m1 = np.array([area @ a[3], area @ a[0]])
    assert np.all(np.abs(m1 - m0) <= 1e-13 * m0), (m1 - m0) / m0
    st = s.stats()
    assert np.allclose(st["mass"], m1, rtol=1e-13)


@pytest.mark.parametrize("case", ["smooth", "translation"])
def test_fp32_l1_error_vs_fp64_oracle(case):
    prob = inputs.smooth_periodic(16) if case == "smooth" else inputs.translation(16)
    (a, gr, tg, st), (ao, go, to) = run_both(prob, 100, precision=FP32)
    area = areas(prob.mesh)
    for v in (0, 3):
        l1 = np.sum(area * np.abs(a[v] - ao[v])) / np.sum(area * np.abs(ao[v]))
        assert l1 <= 1e-5, (v, l1)


def test_fp32_matches_oracle_on_dambreak_all_variables():
    """The FP32 form on the 16^2 interface dam break (60 stages, WENO active
    at the jumps) against the FP64 oracle, every variable and gradient, each
    scaled as the FP64 comparison scales it: area-weighted mean difference
    within 2e-5 and largest within 1e-4 of the scale (measured: at most
    5.7e-6 and 3.1e-5 for the variables, 1.1e-5 and 2.4e-5 for the
    gradients; FP32 deviation arithmetic, ~1e-7 per operation, carried
    through 60 stages of nonlinear weights)."""
    prob = inputs.interface_dambreak(16)
    (a, gr, tg, st), (ao, go, to) = run_both(prob, 60, precision=FP32)
    assert st["status"] == 0
    sa, sg = scales(prob, ao, go)
    area = areas(prob.mesh)
    for v in range(6):
        d = np.abs(a[v] - ao[v]) / sa[v]
        dg = np.abs(gr[v] - go[v]).sum(0) / sg[v]
        assert (area @ d) / area.sum() <= 2e-5 and d.max() <= 1e-4, (v, (area @ d) / area.sum(), d.max())
        assert (area @ dg) / area.sum() <= 5e-5 and dg.max() <= 1e-4 * 2, (v, (area @ dg) / area.sum(), dg.max())


def test_ensemble_instances_match_single_runs():
    probs = [inputs.smooth_periodic(6), inputs.smooth_periodic(9, seed=5), inputs.translation(7)]
    par = g.default_params(g=9.81, chi=0.98, cfl=0.5)
    ens = g.Solver([p.mesh for p in probs], par, np.concatenate([p.b_vert for p in probs]))
    ens.set_state(np.concatenate([p.avg for p in probs], axis=1), np.concatenate([p.grad for p in probs], axis=2))
    ens.advance(8)
    a, gr = ens.get_state()
    off = 0
    for p in probs:
        s = g.Solver(p.mesh, par, p.b_vert)
        s.set_state(p.avg, p.grad)
        s.advance(8)
        b, h = s.get_state()
        n = p.mesh.n_tri
        assert np.array_equal(a[:, off:off + n], b) and np.array_equal(gr[:, :, off:off + n], h)
        off += n


def test_fp64_matches_oracle_at_64sq_with_autotuned_shapes():
    """8,192 triangles (256 reconstruction tiles, many Morton blocks), 20
    stages in the launch shapes the autotuner picks, element by element."""
    prob = inputs.smooth_periodic(64)
    s = g.problem_solver(prob, precision=FP64)
    shapes = s.autotune(1)
    s.set_state(prob.avg, prob.grad)
    s.advance(20)
    a, gr = s.get_state()
    o = Oracle.from_problem(prob)
    o.advance(20)
    ao, go = o.get_state()
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (shapes, ra, rg)


def test_bench_size_properties():
    """At the benchmark's full sizes: the lake at rest (1024^2 squares,
    2,097,152 triangles) in both forms; and the large configuration
    (7,997,584 triangles) after 20 stages in the launch shapes the autotuner
    picks, the FP32 form within 1e-5 (relative L1 of each depth) of the FP64
    form, both conserving each layer's mass to 1e-13."""
    prob = inputs.lake_at_rest(1024)
    for precision in (FP64, FP32):
        s = g.problem_solver(prob, precision=precision)
        s.advance(4)
        a, _ = s.get_state()
        bav = prob.b_vert[prob.mesh.tri].mean(1)
        assert np.abs(a[3] + bav - 0.8).max() <= 1e-12
        assert np.abs(a[[1, 2, 4, 5]]).max() <= 1e-12
        del s
        torch.cuda.empty_cache()
    prob = inputs.internal_wave_ridge()
    area = areas(prob.mesh)
    out = {}
    for precision in (FP64, FP32):
        s = g.problem_solver(prob, precision=precision)
        s.autotune(1)
        s.set_state(prob.avg, prob.grad)
        s.advance(20)
        a, _ = s.get_state()
        assert s.stats()["status"] == 0
        for v in (0, 3):
            assert abs(area @ a[v] - area @ prob.avg[v]) <= 1e-13 * (area @ prob.avg[v])
        out[precision] = a
        del s
        torch.cuda.empty_cache()
    for v in (0, 3):
        l1 = np.sum(area * np.abs(out[FP32][v] - out[FP64][v])) / np.sum(area * np.abs(out[FP64][v]))
        assert l1 <= 1e-5, (v, l1)
