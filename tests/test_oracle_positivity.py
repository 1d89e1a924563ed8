"""The oracle's positivity option (not in the paper, off by default): point
depths held to a floor by scaling a layer's depth and discharge polynomials
toward their averages, and point velocities bounded by the edge's two cells'
average velocities where a layer's point depths dip below half its average.

Pins: where no point depth comes near the floor and none dips that far the
option changes nothing, bit for bit (the exact translation case); the
paper's Riemann problem II (Sec. 4.3), on which the method as read stops in
its first steps with a non-finite interface state, runs to the paper's t = 1
with the option, each layer's mass conserved to rounding, depths within the
initial range widened by the waves' overshoot and the free surface within
2.5% of its initial flat level."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2306_04467_gb300 import inputs


def areas(mesh):
    xy, tri = mesh.xy, mesh.tri
    d1, d2 = xy[tri[:, 1]] - xy[tri[:, 0]], xy[tri[:, 2]] - xy[tri[:, 0]]
    return 0.5 * np.abs(d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0])


def test_option_changes_nothing_on_a_smooth_flow():
    prob = inputs.translation(8)
    out = []
    for floor in (0.0, 0.01):
        o = Oracle.from_problem(prob)
        o.set_positivity(floor)
        o.advance(10 ** 7, t_end=prob.t_end)
        out.append(o.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_riemann_problem_two_runs_with_the_option():
    prob = inputs.riemann_two(8)
    plain = Oracle.from_problem(prob)
    with pytest.raises(RuntimeError):
        plain.advance(10 ** 7, t_end=prob.t_end)
    assert plain.t < 0.05
    o = Oracle.from_problem(prob)
    o.set_positivity(0.01)
    o.advance(10 ** 7, t_end=prob.t_end)
    assert abs(o.t - prob.t_end) < 1e-12
    a, _ = o.get_state()
    area = areas(prob.mesh)
    for v in (0, 3):
        assert abs(area @ a[v] - area @ prob.avg[v]) <= 1e-12 * (area @ prob.avg[v])
    for v in (0, 3):
        assert 0.15 <= a[v].min() and a[v].max() <= 1.85, (v, a[v].min(), a[v].max())
    surface = a[0] + a[3]
    assert np.abs(surface - 2.0).max() <= 0.05, np.abs(surface - 2.0).max()


def point_depths(o, prob, b):
    """Least depth per cell and layer (0: lower h1, 1: upper h2) over the
    cell's edge Gauss points, from the current reconstruction; b(x) is the
    bottom (linear, so its vertex interpolation is exact)."""
    xq, lr = o.edge_points()
    hmin = np.full((prob.mesh.n_tri, 2), np.inf)
    for e in range(xq.shape[0]):
        for q in range(2):
            x, y = xq[e, q]
            for c in lr[e]:
                if c < 0:
                    continue
                v, _ = o.eval(c, x, y)
                hmin[c, 0] = min(hmin[c, 0], v[3] - b(x))
                hmin[c, 1] = min(hmin[c, 1], v[0])
    return hmin


def test_scaling_brings_the_least_point_depth_to_the_floor():
    """The scaling step alone on Riemann problem II's jump over a sloping
    bottom (b = 0.03 x, so the lower layer's level keeps the bottom's linear
    part), after one stage of the method as read (whose reconstruction then
    overshoots to point depths of -0.4 times the average): a layer whose
    least point depth was below f times its average ends with that least
    depth exactly at f times the average; every other layer keeps its
    reconstruction, bit for bit."""
    base = inputs.riemann_two(8)
    b = lambda x: 0.03 * x
    bv = b(base.mesh.xy[:, 0])
    prob = inputs.Problem("riemann_two_slope", base.mesh, bv, base.avg, base.grad, g=base.g, chi=base.chi,
                          cfl=base.cfl, t_end=base.t_end)
    f = 0.3
    o = Oracle.from_problem(prob)
    o.advance(1)
    o.reconstruct()
    before = point_depths(o, prob, b)
    o.set_positivity(f)
    o.positivity_scale()
    after = point_depths(o, prob, b)
    a, _ = o.get_state()
    hbar = np.stack([a[3], a[0]], 1)
    scaled = before < f * hbar
    assert scaled.any() and not scaled.all()
    assert np.allclose(after[scaled], f * hbar[scaled], rtol=0, atol=1e-12)
    assert np.array_equal(after[~scaled], before[~scaled])
