"""Pins of the oracle's troubled-cell gate support (an addition to the paper).

The gate feeds on 24 features of the cell averages and gradients and is
trained on the departure of the WENO weights of Sec. 3.4 from the linear
ones; cells it calls smooth take the linear weights. These tests check the
oracle's features against the same quantities formed from the mesh geometry
for linear data, the weight departure against its limits (zero for linear
data, bounded below by the P3 weight the oracle reports), and the linear
mask against exact cubic reproduction of the P3 least-squares polynomial.
"""
import numpy as np

from oracle import oracle as orc
from paper_2306_04467_gb300 import inputs

from test_oracle_pins import _cubic, _interior_cells


def _polynomial_state(mesh, rng, degree):
    fs = []
    for v in range(6):
        f, fx, fy = _cubic(rng)
        if degree == 1:
            c0, c1, c2 = rng.normal(size=3)
            f = (lambda a, b, c: (lambda x, y: a + b * x + c * y))(c0, c1, c2)
            fx = (lambda b: (lambda x, y: b + 0 * x))(c1)
            fy = (lambda c: (lambda x, y: c + 0 * x))(c2)
        if v in (0, 3):
            f = (lambda g: (lambda x, y: 3.0 + g(x, y)))(f)
        fs.append((f, fx, fy))
    avg = np.stack([inputs.cell_average(f, mesh, 5) for f, _, _ in fs])
    grad = np.stack([np.stack([inputs.cell_average(fx, mesh, 5), inputs.cell_average(fy, mesh, 5)])
                     for _, fx, fy in fs])
    return fs, avg, grad


def _max_error(o, mesh, fs, cells):
    worst = 0.0
    for c in cells:
        P = mesh.xy[mesh.tri[c]]
        for bary in ((0.2, 0.3), (0.6, 0.1), (0.05, 0.9)):
            x, y = P[0] + bary[0] * (P[1] - P[0]) + bary[1] * (P[2] - P[0])
            val, g = o.eval(c, x, y)
            for v, (f, fx, fy) in enumerate(fs):
                worst = max(worst, abs(val[v] - f(x, y)), abs(g[v, 0] - fx(x, y)), abs(g[v, 1] - fy(x, y)))
    return worst


def test_linear_mask_gives_the_p3_polynomial():
    """With every cell masked, the reconstruction is the P3 least-squares fit,
    exact for cubics at the default gamma_H; without the mask it is not."""
    mesh = inputs.jittered_mesh(10, 10, seed=11, bc="wall")
    fs, avg, grad = _polynomial_state(mesh, np.random.default_rng(21), 3)
    o = orc.Oracle(mesh, None)
    o.set_state(avg, grad)
    cells = _interior_cells(mesh, 0.25)
    o.reconstruct()
    assert _max_error(o, mesh, fs, cells) > 1e-6
    o.set_linear_mask(np.ones(mesh.n_tri, np.uint8))
    o.reconstruct()
    assert _max_error(o, mesh, fs, cells) < 1e-9
    assert np.all(o.weight_departure() == 0)
    o.set_linear_mask(None)
    o.reconstruct()
    assert _max_error(o, mesh, fs, cells) > 1e-6


def test_weight_departure_limits():
    # linear data: every candidate is exact, all smoothness indicators agree
    mesh = inputs.jittered_mesh(10, 10, seed=12, bc="wall")
    _, avg, grad = _polynomial_state(mesh, np.random.default_rng(22), 1)
    o = orc.Oracle(mesh, None)
    o.set_state(avg, grad)
    o.reconstruct()
    cells = _interior_cells(mesh, 0.25)
    assert o.weight_departure()[cells].max() <= 1e-10
    # a discontinuous state: the departure bounds that of the P3 weight
    p = inputs.interface_dambreak(24)
    o = orc.Oracle.from_problem(p)
    o.advance(10)
    o.reconstruct()
    d = o.weight_departure()
    om = o.omega()
    assert np.all(np.abs(om / orc.GAMMA_HI - 1) <= d + 1e-15)
    assert d.max() > 0.5 and np.median(d) < 1e-6


def test_gate_features_on_linear_data():
    """For linear eta1 and h2 the features follow from the centroids."""
    mesh = inputs.jittered_mesh(9, 8, domain=(0, 1.2, 0, 1), seed=13, bc="wall")
    rng = np.random.default_rng(23)
    coef = {3: (0.8, 0.3, -0.2), 0: (0.4, -0.1, 0.25)}
    avg = np.zeros((6, mesh.n_tri))
    grad = np.zeros((6, 2, mesh.n_tri))
    P = mesh.xy[mesh.tri]
    cx, cy = P[:, :, 0].mean(1), P[:, :, 1].mean(1)
    for v, (a, b, c) in coef.items():
        avg[v] = a + b * cx + c * cy            # cell average of a linear field
        grad[v, 0], grad[v, 1] = b, c
    avg[[1, 2, 4, 5]] = 0.01 * rng.normal(size=(4, mesh.n_tri))
    o = orc.Oracle(mesh, None)
    o.set_state(avg, grad)
    X = o.gate_features()
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                        - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    # face k of a cell is its edge from vertex k to vertex k + 1
    owner = {}
    for t in range(mesh.n_tri):
        for k in range(3):
            a, b = mesh.tri[t, k], mesh.tri[t, (k + 1) % 3]
            owner.setdefault((min(a, b), max(a, b)), []).append(t)
    cells = _interior_cells(mesh, 0.2)
    assert len(cells) > 30
    for t in cells:
        nb = []
        for k in range(3):
            a, b = mesh.tri[t, k], mesh.tri[t, (k + 1) % 3]
            pair = owner[(min(a, b), max(a, b))]
            nb.append(pair[0] if pair[1] == t else pair[1])
        hs = np.sqrt(area[t])
        for s, v in enumerate((3, 0)):
            q = avg[v, [t] + nb]
            raw = np.zeros(12)
            raw[0::3] = q - q.mean()
            raw[1::3] = hs * coef[v][1]
            raw[2::3] = hs * coef[v][2]
            ref = raw / np.sqrt(np.sum(raw ** 2) + orc.WENO_EPS * area[t] * (1 + q[0] ** 2))
            assert np.abs(X[t, 12 * s:12 * s + 12] - ref).max() <= 1e-13, (t, v)


def test_p3_weight_collapses_at_a_jump_and_is_linear_away_from_it():
    """The nonlinear reconstruction exists to handle discontinuities (Sec. 3.4)
    and the edge weight w of Sec. 2.3 is its P3 weight over the linear one
    (reading R6): on a step in eta1 the cells at the jump keep under a tenth
    of the linear P3 weight, while cells whose stencils see only constant
    data keep exactly the linear weight."""
    mesh = inputs.jittered_mesh(24, 6, domain=(0.0, 1.0, 0.0, 0.25), seed=4, bc="periodic")
    o = orc.Oracle(mesh, None, g=9.81, chi=0.5)
    _, cx, _ = o.geometry()
    avg = np.zeros((6, mesh.n_tri))
    avg[3] = np.where((cx > 0.25) & (cx < 0.75), 0.7, 0.5)
    avg[0] = 0.3
    o.set_state(avg, np.zeros((6, 2, mesh.n_tri)))
    o.reconstruct()
    ratio = o.omega().reshape(mesh.n_tri, 6)[:, 3] / 0.85
    dist = np.minimum(np.abs(cx - 0.25), np.abs(cx - 0.75))
    at, away = dist < 0.03, dist >= 0.1
    assert at.sum() >= 40 and away.sum() >= 150
    assert ratio[at].max() < 0.1
    assert np.abs(ratio[away] - 1).max() < 1e-12
