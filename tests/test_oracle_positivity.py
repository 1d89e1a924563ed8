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
