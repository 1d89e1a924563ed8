"""The seeded input generators against their stated recipe (no scheme
arithmetic lives there): the random stream, the jittered meshes, the
bathymetries, the ensemble sizes and the initial states of the workloads."""
import math

import numpy as np

from paper_2306_04467_gb300 import inputs


def test_splitmix64_matches_its_published_outputs():
    """Seed 0 gives the reference implementation's first four outputs."""
    got = [int(v) for v in inputs.splitmix64(0, 4)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    u = inputs.uniform01(7, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005


def _areas(mesh):
    p = mesh.xy[mesh.tri]
    return 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) -
                  (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))


def test_jittered_mesh_recipe():
    """2 nx ny counter-clockwise triangles tiling the domain; interior
    vertices within 0.15 h of the grid, boundary vertices on the boundary;
    each seed its own diagonals, the same seed the same mesh."""
    nx, ny, dom = 12, 7, (0.0, 1.5, -0.5, 0.5)
    m = inputs.jittered_mesh(nx, ny, domain=dom, seed=5, bc="wall")
    a = _areas(m)
    assert m.n_tri == 2 * nx * ny and a.min() > 0
    assert abs(a.sum() - 1.5 * 1.0) < 1e-12
    hx, hy = 1.5 / nx, 1.0 / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    gx, gy = dom[0] + ii.ravel() * hx, dom[2] + jj.ravel() * hy
    assert np.abs(m.xy[:, 0] - gx).max() <= 0.15 * hx + 1e-15
    assert np.abs(m.xy[:, 1] - gy).max() <= 0.15 * hy + 1e-15
    edge = (ii.ravel() == 0) | (ii.ravel() == nx) | (jj.ravel() == 0) | (jj.ravel() == ny)
    assert np.array_equal(m.xy[edge], np.stack([gx, gy], 1)[edge])
    again = inputs.jittered_mesh(nx, ny, domain=dom, seed=5, bc="wall")
    other = inputs.jittered_mesh(nx, ny, domain=dom, seed=6, bc="wall")
    assert np.array_equal(again.xy, m.xy) and np.array_equal(again.tri, m.tri)
    assert not np.array_equal(other.tri, m.tri)
    p = inputs.jittered_mesh(nx, ny, domain=dom, seed=5, bc="periodic")
    assert p.period == (1.5, 1.0) and (p.tri_bc == inputs.BC_PERIODIC).sum() == 2 * (nx + ny)


def test_fourier_bathymetry_is_bounded_and_periodic():
    """Eight modes with wavenumbers in {1..4}^2 and amplitudes summing to 0.2."""
    b = inputs.fourier_bathymetry(seed=3)
    x, y = np.meshgrid(np.linspace(0, 1, 101), np.linspace(0, 1, 101))
    v = b(x, y)
    assert np.abs(v).max() <= 0.2 + 1e-12 and np.abs(v).max() > 0.02
    assert np.abs(b(x + 1.0, y) - v).max() < 1e-12 and np.abs(b(x, y + 1.0) - v).max() < 1e-12


def test_ensemble_sizes_are_log_uniform_square_meshes():
    n = inputs.ensemble_sizes(256)
    nt = 2 * n * n
    assert nt.min() >= 2 * round(math.sqrt(5000 / 2)) ** 2 * 0.9 and nt.max() <= 200000 * 1.02
    # log-uniform on [5k, 200k]: the median of log(N_T) near the log of the geometric mean
    assert abs(np.median(np.log(nt)) - 0.5 * (math.log(5000) + math.log(200000))) < 0.3
    assert np.array_equal(n, inputs.ensemble_sizes(256))


def test_workload_initial_states():
    """The lake at rest has a flat interface (h1 + B = 0.8 per cell, B its
    cell average), h2 = 0.2 and no motion; the interface dam break carries
    (h1, h2) = (0.6, 0.4) left of x = 0 and (0.4, 0.6) right of it."""
    p = inputs.lake_at_rest(16)
    bavg = p.b_vert[p.mesh.tri].mean(1)
    assert np.abs(p.avg[3] + bavg - 0.8).max() < 1e-14 and np.all(p.avg[0] == 0.2)
    assert np.all(p.avg[[1, 2, 4, 5]] == 0)
    d = inputs.interface_dambreak(12)
    cx = d.mesh.xy[d.mesh.tri].mean(1)[:, 0]
    far = np.abs(cx) > 0.2
    assert np.allclose(d.avg[3][far], np.where(cx[far] < 0, 0.6, 0.4), atol=1e-14)
    assert np.allclose(d.avg[0][far], np.where(cx[far] < 0, 0.4, 0.6), atol=1e-14)
    assert np.abs(d.avg[3] + d.avg[0] - 1.0).max() < 1e-14
