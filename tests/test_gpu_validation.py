"""The paper's Riemann problem I (Sec. 4.3) and channel flow over a non-flat
bottom (Sec. 4.5) as smoke tests on the GPU, and Riemann problem II (Sec.
4.3) and the circular interface (Sec. 4.6) with the positivity option (not
in the paper; the method as read reaches a vacuum at an interface state in
their first steps).

The paper compares them with reference solutions from other papers by plot
only, so the checks are what the physics fixes: each layer's mass is
conserved, for Riemann problem I h1 keeps its initial value ahead of the
fastest wave and behind the slowest up to the scheme's precursor (the bound
the oracle pin holds), for the channel flow the depths stay positive and
the free surface near flat, and the FP64 form matches the oracle element by
element on a coarse version of each. (Riemann problem II and the circular interface, whose 0.2 |
1.8 jumps make the reconstruction's point depths negative in the first
stage with the method as read, are recorded with the design notes.)
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2306_04467_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2306_04467_gb300 import gks2l as g  # noqa: E402

from test_gpu_parity import areas, max_rel  # noqa: E402


def advance_to(s, t_end, chunk=200):
    """Advance to t_end in chunks of stages (gks2l_advance enqueues every
    stage it is asked for; steps past t_end compute nothing new)."""
    while True:
        t = s.advance(chunk, t_end=t_end)
        if t >= t_end * (1 - 1e-12):
            return t


def run(prob, precision, t_end=None, **kw):
    s = g.problem_solver(prob, precision=precision, **kw)
    advance_to(s, prob.t_end if t_end is None else t_end)
    a, gr = s.get_state()
    assert s.stats()["status"] == 0
    return a, gr


def masses_kept(prob, a, rtol=1e-12):
    area = areas(prob.mesh)
    for v in (0, 3):
        m0, m1 = area @ prob.avg[v], area @ a[v]
        assert abs(m1 - m0) <= rtol * m0, (v, (m1 - m0) / m0)


def centroids(mesh):
    return mesh.xy[mesh.tri].mean(1)


def test_fp64_matches_oracle_on_riemann_problem_one():
    """ΔX = 1/25 to the paper's t = 0.1, element by element against the oracle."""
    prob, t = inputs.riemann_one(25), 0.1
    a, gr = run(prob, g.GKS2L_FP64, t)
    o = Oracle.from_problem(prob)
    o.advance(10 ** 7, t_end=t)
    ao, go = o.get_state()
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (ra, rg)


def departure(prob, a):
    c = centroids(prob.mesh)
    ahead = (c[:, 0] > 0.95) & (c[:, 0] < 1.7)
    behind = (c[:, 0] > 0.05) & (c[:, 0] < 0.2)
    return max(np.abs(a[3][ahead] - 0.55).max(), np.abs(a[3][behind] - 0.5).max())


def test_riemann_problem_one_fp64():
    """At the paper's ΔX = 1/100 and at 1/200: h1's departure ahead of the
    fastest wave and behind the slowest within the oracle pin's 3e-4 at
    1/100 and shrinking with the mesh; masses kept."""
    dep = []
    for n in (100, 200):
        prob = inputs.riemann_one(n)
        a, _ = run(prob, g.GKS2L_FP64)
        masses_kept(prob, a)
        dep.append(departure(prob, a))
    print("riemann I departure (FP64)", dep)
    assert dep[0] <= 3e-4 and dep[1] < dep[0], dep


def test_riemann_problem_one_fp32():
    """The FP32 form at the paper's ΔX = 1/100: the same bound, masses kept.
    (At 1/200 the FP32 form's rounding seeds the strong-advection mode left
    open at chi >= 0.97 and the departure reaches 2.4e-3; recorded with the
    design notes.)"""
    prob = inputs.riemann_one(100)
    a, _ = run(prob, g.GKS2L_FP32)
    masses_kept(prob, a)
    dep = departure(prob, a)
    print("riemann I departure (FP32)", dep)
    assert dep <= 3e-4, dep


def test_fp64_matches_oracle_on_channel_flow():
    """Channel flow at 40 x 10 squares to the paper's t = 0.1, element by
    element against the oracle."""
    prob = inputs.channel_flow(40)
    a, gr = run(prob, g.GKS2L_FP64)
    o = Oracle.from_problem(prob)
    o.advance(10 ** 7, t_end=prob.t_end)
    ao, go = o.get_state()
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (ra, rg)


def test_channel_flow_at_the_papers_mesh():
    """At the paper's cell size 1/200 to t = 0.1 (the interface still
    smooth): masses kept in both forms, depths positive, the free surface
    within 2.5% of its initial 1.2 while the interface over the bump moves
    by about 10%, and the FP32 form within 1e-5 (L1, relative) of the FP64
    form."""
    prob = inputs.channel_flow(200)
    bav = prob.b_vert[prob.mesh.tri].mean(1)
    out = {}
    for prec in (g.GKS2L_FP64, g.GKS2L_FP32):
        a, _ = run(prob, prec)
        masses_kept(prob, a)
        assert a[3].min() > 0 and a[0].min() > 0
        surface = a[3] + a[0] + bav
        assert np.abs(surface - 1.2).max() <= 0.03, np.abs(surface - 1.2).max()
        out[prec] = a
    eta = out[g.GKS2L_FP64][3] + bav
    assert eta.max() - eta.min() >= 0.05, (eta.min(), eta.max())
    area = areas(prob.mesh)
    l1 = max(area @ np.abs(out[g.GKS2L_FP32][v] - out[g.GKS2L_FP64][v]) / (area @ np.abs(out[g.GKS2L_FP64][v]))
             for v in (0, 1, 3, 4))
    print("channel flow FP32 vs FP64 L1", l1)
    assert l1 <= 1e-5, l1


FLOOR = 0.01   # the positivity option's depth floor, a fraction of the cell average


@pytest.mark.parametrize("case", ["riemann_two", "circular_interface"])
def test_fp64_matches_oracle_with_positivity(case):
    """Riemann problem II at 80 x 8 squares to t = 1 and the circular
    interface at 30 x 30 squares to t = 4, with the option, element by
    element against the oracle with the same option."""
    prob = inputs.riemann_two(8) if case == "riemann_two" else inputs.circular_interface(3)
    a, gr = run(prob, g.GKS2L_FP64, positivity_floor=FLOOR)
    o = Oracle.from_problem(prob)
    o.set_positivity(FLOOR)
    o.advance(10 ** 7, t_end=prob.t_end)
    ao, go = o.get_state()
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (ra, rg)


@pytest.mark.parametrize("precision", [g.GKS2L_FP64, g.GKS2L_FP32])
def test_riemann_problem_two_with_positivity(precision):
    """At the paper's cell size 1/40 to t = 1: masses kept, both depths
    within [0.15, 1.85] (the initial 0.2 and 1.8 widened by the waves'
    overshoot) and the free surface within 6% of its initial level 2 (the
    release sends out surface waves: 4.8% at this mesh in both forms)."""
    prob = inputs.riemann_two(40)
    a, _ = run(prob, precision, positivity_floor=FLOOR)
    masses_kept(prob, a)
    for v in (0, 3):
        assert 0.15 <= a[v].min() and a[v].max() <= 1.85, (v, a[v].min(), a[v].max())
    assert np.abs(a[0] + a[3] - 2.0).max() <= 0.12


@pytest.mark.parametrize("precision", [g.GKS2L_FP64, g.GKS2L_FP32])
def test_circular_interface_with_positivity(precision):
    """At the paper's cell size 1/10 to t = 4: masses kept, depths positive,
    the free surface within 5% of flat, and the collapse as round as the
    mesh allows: the lower layer's mass in the four quadrants about the
    circle's centre within 3% of each other (cells cut by the quadrant lines
    alone give 1% at the start; the oracle's spread falls from 6.4% to 3.9%
    between 3 and 4 squares per unit)."""
    prob = inputs.circular_interface(10)
    a, _ = run(prob, precision, positivity_floor=FLOOR)
    masses_kept(prob, a)
    assert a[0].min() > 0 and a[3].min() > 0
    assert np.abs(a[0] + a[3] - 2.0).max() <= 0.1
    c = centroids(prob.mesh) - 5.0
    area = areas(prob.mesh)
    quad = [(c[:, 0] >= 0) & (c[:, 1] >= 0), (c[:, 0] < 0) & (c[:, 1] >= 0),
            (c[:, 0] < 0) & (c[:, 1] < 0), (c[:, 0] >= 0) & (c[:, 1] < 0)]
    m = np.array([area[q] @ a[3][q] for q in quad])
    assert (m.max() - m.min()) <= 0.03 * m.mean(), m
