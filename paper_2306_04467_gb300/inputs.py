"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module generates meshes, bathymetry and initial cell data only; it holds
none of the scheme's arithmetic (no reconstruction, no flux, no source, no time
stepping). Every random number comes from splitmix64 (Steele, Lea & Flood 2014),
vectorised over a counter, so a (seed, size) pair fixes the whole input.

Meshes are N_x x N_y squares over a rectangle, each square split along one of
its diagonals chosen by a seeded coin, with the interior vertices jittered
uniformly by +-0.15 of the square size in each coordinate (boundary vertices
stay on the boundary lines, so wall edges stay straight and periodic images
match exactly).

State layout used everywhere: 6 variables per cell in the paper's order
(Sec. 2.1, Eq. SWE-macro):  h2, h2*U2, h2*V2, h1, h1*U1, h1*V1, with layer 1
the lower layer and layer 2 the upper one. Arrays are variable-major:
avg[v, j] and grad[v, d, j] (d = 0 for x, 1 for y).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_INTERIOR = 0
BC_WALL = 1
BC_PERIODIC = 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of splitmix64 started at `seed`, counter positions offset+1..offset+n."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by the Box-Muller transform of two uniform streams."""
    u1 = uniform01(seed, n, offset)
    u2 = uniform01(seed ^ 0x5DEECE66D, n, offset)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclasses.dataclass
class Mesh:
    """A triangle mesh as the C ABI takes it.

    xy      (n_vert, 2) float64 vertex coordinates
    tri     (n_tri, 3) int32 vertex indices, counter-clockwise
    tri_bc  (n_tri, 3) int8: kind of the edge from tri[:, k] to tri[:, (k+1)%3]
            (BC_INTERIOR, BC_WALL or BC_PERIODIC)
    period  (px, py): translation that maps one periodic boundary onto the
            opposite one (0 where a direction is not periodic)
    """
    xy: np.ndarray
    tri: np.ndarray
    tri_bc: np.ndarray
    period: tuple
    nx: int = 0
    ny: int = 0
    domain: tuple = (0.0, 1.0, 0.0, 1.0)

    @property
    def n_vert(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])


def jittered_mesh(nx: int, ny: int, domain=(0.0, 1.0, 0.0, 1.0), seed: int = 1,
                  jitter: float = 0.15, bc: str = "periodic") -> Mesh:
    """nx x ny squares, each cut along a seeded diagonal, interior vertices jittered.

    bc: "periodic" (both directions) or "wall" (all four sides).
    """
    x0, x1, y0, y1 = (float(v) for v in domain)
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    nvx, nvy = nx + 1, ny + 1
    nv = nvx * nvy
    ii, jj = np.meshgrid(np.arange(nvx), np.arange(nvy), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    X = x0 + ii * hx
    Y = y0 + jj * hy
    r = uniform01(seed, 2 * nv + nx * ny)
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
    X = np.where(interior, X + (2.0 * r[:nv] - 1.0) * jitter * hx, X)
    Y = np.where(interior, Y + (2.0 * r[nv:2 * nv] - 1.0) * jitter * hy, Y)
    # boundary vertices sit exactly on the boundary lines
    X = np.where(ii == nx, x1, X)
    Y = np.where(jj == ny, y1, Y)
    coin = r[2 * nv:]

    si, sj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    si = si.ravel()
    sj = sj.ravel()
    v00 = sj * nvx + si
    v10 = v00 + 1
    v01 = v00 + nvx
    v11 = v01 + 1
    diag = coin < 0.5
    # diag: cut v00-v11 -> (v00,v10,v11), (v00,v11,v01); else cut v10-v01 -> (v00,v10,v01), (v10,v11,v01)
    t1 = np.where(diag[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(diag[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    tri = np.empty((2 * nx * ny, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2

    kind = BC_PERIODIC if bc == "periodic" else BC_WALL
    ti = ii[tri]
    tj = jj[tri]
    tri_bc = np.zeros(tri.shape, dtype=np.int8)
    for k in range(3):
        a, b = k, (k + 1) % 3
        on = ((ti[:, a] == 0) & (ti[:, b] == 0)) | ((ti[:, a] == nx) & (ti[:, b] == nx)) | \
             ((tj[:, a] == 0) & (tj[:, b] == 0)) | ((tj[:, a] == ny) & (tj[:, b] == ny))
        tri_bc[on, k] = kind
    period = (x1 - x0, y1 - y0) if bc == "periodic" else (0.0, 0.0)
    return Mesh(xy=np.stack([X, Y], 1).astype(np.float64), tri=tri, tri_bc=tri_bc,
                period=period, nx=nx, ny=ny, domain=(x0, x1, y0, y1))


# ---------------------------------------------------------------------------
# quadrature of analytic fields (used to turn formulas into cell data)
# ---------------------------------------------------------------------------

def _gauss_legendre01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(n: int = 4):
    """Collapsed (Duffy) tensor Gauss rule on the reference triangle
    {a, b >= 0, a + b <= 1}: barycentric weights (a, b) and weights summing to 1."""
    s, ws = _gauss_legendre01(n)
    t, wt = _gauss_legendre01(n)
    S, T = np.meshgrid(s, t, indexing="ij")
    W = np.outer(ws, wt) * (1.0 - S)
    a = S.ravel()
    b = (T * (1.0 - S)).ravel()
    w = W.ravel()
    return a, b, w / w.sum()


def cell_points(mesh: Mesh, n: int = 4):
    """Quadrature points (n_tri, nq, 2) and normalised weights (nq,) per cell."""
    a, b, w = triangle_rule(n)
    P = mesh.xy[mesh.tri]  # (nt, 3, 2)
    p0, p1, p2 = P[:, 0], P[:, 1], P[:, 2]
    pts = p0[:, None, :] + a[None, :, None] * (p1 - p0)[:, None, :] + b[None, :, None] * (p2 - p0)[:, None, :]
    return pts, w


def cell_average(f, mesh: Mesh, n: int = 4) -> np.ndarray:
    pts, w = cell_points(mesh, n)
    vals = f(pts[..., 0], pts[..., 1])
    return vals @ w


def p1_average_and_gradient(values_at_vertices: np.ndarray, mesh: Mesh):
    """Cell average and gradient of the continuous piecewise-linear interpolant
    of vertex data (how a vertex-sampled field is turned into cell data)."""
    P = mesh.xy[mesh.tri]
    f = values_at_vertices[mesh.tri]
    avg = f.mean(axis=1)
    d1 = P[:, 1] - P[:, 0]
    d2 = P[:, 2] - P[:, 0]
    df1 = f[:, 1] - f[:, 0]
    df2 = f[:, 2] - f[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    gx = (df1 * d2[:, 1] - df2 * d1[:, 1]) / det
    gy = (df2 * d1[:, 0] - df1 * d2[:, 0]) / det
    return avg, np.stack([gx, gy], 0)


def vertex_samples(f, mesh: Mesh) -> np.ndarray:
    """f at the vertices; on periodic meshes the duplicated boundary vertices
    take the value of their periodic image so the sampled field is single-valued."""
    x = mesh.xy[:, 0].copy()
    y = mesh.xy[:, 1].copy()
    x0, x1, y0, y1 = mesh.domain
    if mesh.period[0] > 0:
        x = np.where(x >= x1, x0, x)
    if mesh.period[1] > 0:
        y = np.where(y >= y1, y0, y)
    return f(x, y)


@dataclasses.dataclass
class Problem:
    """A complete synthetic problem: mesh, vertex bathymetry, parameters and the
    initial cell averages / average gradients (variable-major)."""
    name: str
    mesh: Mesh
    b_vert: np.ndarray
    avg: np.ndarray       # (6, n_tri)
    grad: np.ndarray      # (6, 2, n_tri)
    g: float = 9.81
    chi: float = 0.98
    cfl: float = 0.5
    eps: float = 0.05
    eps_num: float = 5.0
    t_end: float = 0.0
    exact: object = None  # optional callable t -> (avg, grad) of the exact solution


def _fields_to_state(mesh, h2, h2x, h2y, h1, h1x, h1y, u2, v2, u1, v1, n=4):
    """Averages and average gradients from analytic depths/derivatives and
    constant layer velocities."""
    avg = np.zeros((6, mesh.n_tri))
    grad = np.zeros((6, 2, mesh.n_tri))
    A2 = cell_average(h2, mesh, n)
    A1 = cell_average(h1, mesh, n)
    G2 = np.stack([cell_average(h2x, mesh, n), cell_average(h2y, mesh, n)])
    G1 = np.stack([cell_average(h1x, mesh, n), cell_average(h1y, mesh, n)])
    for base, A, G, u, v in ((0, A2, G2, u2, v2), (3, A1, G1, u1, v1)):
        avg[base] = A
        avg[base + 1] = u * A
        avg[base + 2] = v * A
        grad[base] = G
        grad[base + 1] = u * G
        grad[base + 2] = v * G
    return avg, grad


def smooth_periodic(n: int = 16, seed: int = 2306, quad: int = 6) -> Problem:
    """Smooth periodic two-layer flow on the unit square (512 triangles at n=16):
    b = 0.1 sin(2 pi x) cos(2 pi y); h1 = 1 + 0.05 sin(2 pi (x + y)) (lower layer);
    h2 = 1 - b (upper layer); u = v = 0.1 in both layers; g = 9.81, chi = 0.98."""
    mesh = jittered_mesh(n, n, seed=seed, bc="periodic")
    tp = 2.0 * math.pi
    b = lambda x, y: 0.1 * np.sin(tp * x) * np.cos(tp * y)
    h1 = lambda x, y: 1.0 + 0.05 * np.sin(tp * (x + y))
    h1x = lambda x, y: 0.05 * tp * np.cos(tp * (x + y))
    h2 = lambda x, y: 1.0 - b(x, y)
    h2x = lambda x, y: -0.1 * tp * np.cos(tp * x) * np.cos(tp * y)
    h2y = lambda x, y: 0.1 * tp * np.sin(tp * x) * np.sin(tp * y)
    avg, grad = _fields_to_state(mesh, h2, h2x, h2y, h1, h1x, h1x, 0.1, 0.1, 0.1, 0.1, quad)
    return Problem("smooth_periodic", mesh, vertex_samples(b, mesh), avg, grad,
                   g=9.81, chi=0.98, cfl=0.5, t_end=0.05)


def lake_at_rest(n: int = 64, seed: int = 2307, domain=(0.0, 1.0, 0.0, 1.0),
                 amp: float = 0.5, width: float = 50.0, eta1: float = 0.8, h2: float = 0.2,
                 chi: float = 0.98) -> Problem:
    """Two-layer lake at rest over a Gaussian bump, walls on all sides:
    b = amp exp(-width ((x-xc)^2 + (y-yc)^2)), interface h1 + b = eta1 and
    h2 = const, zero velocity. The bathymetry is sampled at the vertices and
    h1 = eta1 - (piecewise-linear b), so the initial interface is exactly flat."""
    mesh = jittered_mesh(n, n, domain=domain, seed=seed, bc="wall")
    xc = 0.5 * (domain[0] + domain[1])
    yc = 0.5 * (domain[2] + domain[3])
    b = lambda x, y: amp * np.exp(-width * ((x - xc) ** 2 + (y - yc) ** 2))
    bv = vertex_samples(b, mesh)
    bavg, bgrad = p1_average_and_gradient(bv, mesh)
    avg = np.zeros((6, mesh.n_tri))
    grad = np.zeros((6, 2, mesh.n_tri))
    avg[0] = h2
    avg[3] = eta1 - bavg
    grad[3] = -bgrad
    return Problem("lake_at_rest", mesh, bv, avg, grad, g=9.81, chi=chi, cfl=0.5)


def translation(n: int = 32, seed: int = 2308, t_end: float = 0.05, quad: int = 6) -> Problem:
    """Periodic analogue of the paper's accuracy test (Sec. 4.1): chi = 1,
    h1 = 0.9 + 0.02 sin(2 pi x) sin(2 pi y), h2 = 1 - h1, U = V = 1 in both
    layers, flat bottom. With chi = 1 and h1 + h2 = const the exact solution is
    pure translation with velocity (1, 1)."""
    mesh = jittered_mesh(n, n, seed=seed, bc="periodic")
    tp = 2.0 * math.pi

    def state_at(t):
        h1 = lambda x, y: 0.9 + 0.02 * np.sin(tp * (x - t)) * np.sin(tp * (y - t))
        h1x = lambda x, y: 0.02 * tp * np.cos(tp * (x - t)) * np.sin(tp * (y - t))
        h1y = lambda x, y: 0.02 * tp * np.sin(tp * (x - t)) * np.cos(tp * (y - t))
        h2 = lambda x, y: 1.0 - h1(x, y)
        h2x = lambda x, y: -h1x(x, y)
        h2y = lambda x, y: -h1y(x, y)
        return _fields_to_state(mesh, h2, h2x, h2y, h1, h1x, h1y, 1.0, 1.0, 1.0, 1.0, quad)

    avg, grad = state_at(0.0)
    return Problem("translation", mesh, np.zeros(mesh.n_vert), avg, grad,
                   g=9.81, chi=1.0, cfl=0.5, t_end=t_end, exact=state_at)


def interface_dambreak(n: int = 895, seed: int = 2309, quad: int = 3) -> Problem:
    """Two-layer interface dam break on [-1, 1]^2 with walls: (h1, h2) = (0.6, 0.4)
    for x < 0 and (0.4, 0.6) for x >= 0, flat bottom, zero velocity, chi = 0.98.
    Cell data are exact averages of the step (area fraction left of x = 0)."""
    mesh = jittered_mesh(n, n, domain=(-1.0, 1.0, -1.0, 1.0), seed=seed, bc="wall")
    left = cell_average(lambda x, y: (x < 0.0).astype(np.float64), mesh, 8)
    avg = np.zeros((6, mesh.n_tri))
    grad = np.zeros((6, 2, mesh.n_tri))
    avg[3] = 0.6 * left + 0.4 * (1.0 - left)
    avg[0] = 0.4 * left + 0.6 * (1.0 - left)
    return Problem("interface_dambreak", mesh, np.zeros(mesh.n_vert), avg, grad,
                   g=9.81, chi=0.98, cfl=0.5)


def fourier_bathymetry(seed: int, n_modes: int = 8, total_amp: float = 0.2):
    """b(x, y) = sum_m a_m cos(2 pi (k_m . x) + phi_m) with k_m in {1..4}^2 and
    sum |a_m| <= total_amp (periodic on the unit square)."""
    r = uniform01(seed, 4 * n_modes)
    kx = 1 + np.floor(4 * r[0:n_modes]).astype(int)
    ky = 1 + np.floor(4 * r[n_modes:2 * n_modes]).astype(int)
    phi = 2.0 * math.pi * r[2 * n_modes:3 * n_modes]
    a = r[3 * n_modes:]
    a = total_amp * a / a.sum()
    tp = 2.0 * math.pi

    def b(x, y):
        out = np.zeros_like(x, dtype=np.float64)
        for m in range(n_modes):
            out = out + a[m] * np.cos(tp * (kx[m] * x + ky[m] * y) + phi[m])
        return out
    return b


def ensemble_sizes(n_inst: int = 256, lo: int = 5000, hi: int = 200000, seed: int = 2310):
    """Seeded log-uniform triangle counts, rounded to square meshes N x N x 2."""
    r = uniform01(seed, n_inst)
    nt = np.exp(np.log(lo) + r * (np.log(hi) - np.log(lo)))
    return np.maximum(8, np.rint(np.sqrt(nt / 2.0)).astype(int))


def ensemble_member(n: int, seed: int, smooth_passes: int = 4) -> Problem:
    """One ensemble instance on the periodic unit square: Fourier bathymetry
    (8 modes, amplitude <= 0.2), interface eta1 = 0.5 + delta with delta a
    0.02 N(0,1) per-cell field smoothed by neighbour averaging over edges,
    free surface at 1 (h1 = eta1 - b, h2 = 1 - eta1), zero velocity, chi = 0.98."""
    mesh = jittered_mesh(n, n, seed=seed, bc="periodic")
    b = fourier_bathymetry(seed ^ 0xB00)
    bv = vertex_samples(b, mesh)
    bavg, bgrad = p1_average_and_gradient(bv, mesh)
    delta = 0.02 * normal01(seed ^ 0xD17A, mesh.n_tri)
    # smoothing by averaging with the cells that share a vertex index pair
    # (input preparation only; plain graph smoothing over shared edges)
    tri = mesh.tri.astype(np.int64)
    nvx = n + 1
    # identify periodic duplicate vertices so smoothing wraps around
    vx = tri % nvx
    vy = tri // nvx
    vid = (vx % n) + n * (vy % n)
    ekeys = []
    cells = []
    for k in range(3):
        a_, b_ = vid[:, k], vid[:, (k + 1) % 3]
        ekeys.append(np.minimum(a_, b_) * (n * n) + np.maximum(a_, b_))
        cells.append(np.arange(mesh.n_tri))
    ekeys = np.concatenate(ekeys)
    cells = np.concatenate(cells)
    order = np.argsort(ekeys, kind="stable")
    ek = ekeys[order]
    cc = cells[order]
    same = ek[1:] == ek[:-1]
    ca = cc[:-1][same]
    cb = cc[1:][same]
    for _ in range(smooth_passes):
        acc = delta.copy()
        cnt = np.ones_like(delta)
        np.add.at(acc, ca, delta[cb])
        np.add.at(acc, cb, delta[ca])
        np.add.at(cnt, ca, 1.0)
        np.add.at(cnt, cb, 1.0)
        delta = acc / cnt
    eta1 = 0.5 + delta
    avg = np.zeros((6, mesh.n_tri))
    grad = np.zeros((6, 2, mesh.n_tri))
    avg[3] = eta1 - bavg
    grad[3] = -bgrad
    avg[0] = 1.0 - eta1
    return Problem("ensemble_member", mesh, bv, avg, grad, g=9.81, chi=0.98, cfl=0.5)


def internal_wave_ridge(nx: int = 5656, ny: int = 707, seed: int = 2311, quad: int = 3) -> Problem:
    """Internal wave over a ridge on [0, 8] x [0, 1] with walls:
    b = 0.3 exp(-20 (x - 4)^2); interface eta1 = 0.7 - 0.1 exp(-20 (x - 1)^2);
    free surface at 1 (h2 = 1 - eta1); zero velocity; chi = 0.97."""
    mesh = jittered_mesh(nx, ny, domain=(0.0, 8.0, 0.0, 1.0), seed=seed, bc="wall")
    b = lambda x, y: 0.3 * np.exp(-20.0 * (x - 4.0) ** 2)
    bv = vertex_samples(b, mesh)
    bavg, bgrad = p1_average_and_gradient(bv, mesh)
    eta = lambda x, y: 0.7 - 0.1 * np.exp(-20.0 * (x - 1.0) ** 2)
    etax = lambda x, y: 4.0 * (x - 1.0) * np.exp(-20.0 * (x - 1.0) ** 2)
    zero = lambda x, y: np.zeros_like(x)
    avg = np.zeros((6, mesh.n_tri))
    grad = np.zeros((6, 2, mesh.n_tri))
    eavg = cell_average(eta, mesh, quad)
    egx = cell_average(etax, mesh, quad)
    avg[3] = eavg - bavg
    grad[3, 0] = egx - bgrad[0]
    grad[3, 1] = -bgrad[1]
    avg[0] = 1.0 - eavg
    grad[0, 0] = -egx
    del zero
    return Problem("internal_wave_ridge", mesh, bv, avg, grad, g=9.81, chi=0.97, cfl=0.5)


def _two_states(mesh, inside, left, right, quad=8):
    """Cell averages of a two-state layer split: (h1, h2) = left where
    inside(x, y), right elsewhere (exact area fractions by quadrature), zero
    velocity and gradients."""
    frac = cell_average(lambda x, y: inside(x, y).astype(np.float64), mesh, quad)
    avg = np.zeros((6, mesh.n_tri))
    avg[3] = left[0] * frac + right[0] * (1.0 - frac)
    avg[0] = left[1] * frac + right[1] * (1.0 - frac)
    return avg, np.zeros((6, 2, mesh.n_tri))


def riemann_one(n: int = 100, ny: int = 4, seed: int = 7) -> Problem:
    """The paper's Riemann problem I (Sec. 4.3): (h1, h2) = (0.5, 0.5) left of
    the jump and (0.55, 0.45) right of it, U = 2.5 in both layers, chi = 0.98,
    G = 10, t = 0.1, on squares of side 1/n. A periodic strip [0, 3] x
    [0, ny/n] stands in for the paper's [0, 1] x [0, 0.5]: the jump at x = 0.3
    and a mirrored one at x = 1.8, whose waves cannot reach the first one's
    region by t = 0.1."""
    mesh = jittered_mesh(3 * n, ny, domain=(0.0, 3.0, 0.0, ny / n), seed=seed, bc="periodic")
    avg, grad = _two_states(mesh, lambda x, y: (x >= 0.3) & (x < 1.8), (0.55, 0.45), (0.5, 0.5))
    avg[4], avg[1] = 2.5 * avg[3], 2.5 * avg[0]
    return Problem("riemann_one", mesh, np.zeros(mesh.n_vert), avg, grad, g=10.0, chi=0.98, cfl=0.5, t_end=0.1)


def riemann_two(n: int = 40, seed: int = 8) -> Problem:
    """The paper's Riemann problem II (Sec. 4.3): (h1, h2) = (0.2, 1.8) for
    x < 5 and (1.8, 0.2) for x >= 5 on [0, 10] x [0, 1], zero velocity,
    chi = 0.98, G = 9.81, t = 1, squares of side 1/n. Walls close the ends,
    which no wave reaches by t = 1."""
    mesh = jittered_mesh(10 * n, n, domain=(0.0, 10.0, 0.0, 1.0), seed=seed, bc="wall")
    avg, grad = _two_states(mesh, lambda x, y: x < 5.0, (0.2, 1.8), (1.8, 0.2))
    return Problem("riemann_two", mesh, np.zeros(mesh.n_vert), avg, grad, g=9.81, chi=0.98, cfl=0.5, t_end=1.0)


def circular_interface(n: int = 10, seed: int = 9) -> Problem:
    """The paper's 2-D interface propagation (Sec. 4.6): (h1, h2) = (1.8, 0.2)
    inside the circle of radius 2 about (5, 5) and (0.2, 1.8) outside, on
    [0, 10]^2, zero velocity, chi = 0.98, G = 9.81, run to t = 4, squares of
    side 1/n. Walls stand in for the paper's free boundaries: the surface is
    flat at the start and the interface's waves stay far from the sides."""
    mesh = jittered_mesh(10 * n, 10 * n, domain=(0.0, 10.0, 0.0, 10.0), seed=seed, bc="wall")
    avg, grad = _two_states(mesh, lambda x, y: (x - 5.0) ** 2 + (y - 5.0) ** 2 < 4.0, (1.8, 0.2), (0.2, 1.8))
    return Problem("circular_interface", mesh, np.zeros(mesh.n_vert), avg, grad, g=9.81, chi=0.98, cfl=0.5,
                   t_end=4.0)


def channel_flow(n: int = 200, seed: int = 10) -> Problem:
    """The paper's channel flow over a non-flat bottom (Sec. 4.5): b =
    0.5 exp(-100 (x - 0.5)^2), h1 = 0.8 - b, h2 = 0.4, U1 = -0.2, U2 = 0.15,
    V = 0, on [0, 1] x [0, 0.25] with squares of side 1/n, t = 0.1. The paper
    names no density ratio or gravity for this case: chi = 0.98 and G = 9.81,
    as in its neighbouring cases. The mesh is periodic: across the channel
    that equals the paper's walls for this y-independent flow with V = 0,
    and along it the periodic ends stand in for the paper's free ones until
    t = 0.1 (the fastest wave, about 3.6, travels 0.36 from where the bottom
    slopes, and the bottom is 7e-12 at the ends). The bathymetry is sampled
    at the vertices and h1 = 0.8 - (piecewise-linear b)."""
    mesh = jittered_mesh(n, n // 4, domain=(0.0, 1.0, 0.0, 0.25), seed=seed, bc="periodic")
    b = lambda x, y: 0.5 * np.exp(-100.0 * (x - 0.5) ** 2)
    bv = vertex_samples(b, mesh)
    bavg, bgrad = p1_average_and_gradient(bv, mesh)
    avg = np.zeros((6, mesh.n_tri))
    grad = np.zeros((6, 2, mesh.n_tri))
    avg[3] = 0.8 - bavg
    grad[3] = -bgrad
    avg[4] = -0.2 * avg[3]
    grad[4] = -0.2 * grad[3]
    avg[0] = 0.4
    avg[1] = 0.15 * 0.4
    return Problem("channel_flow", mesh, bv, avg, grad, g=9.81, chi=0.98, cfl=0.5, t_end=0.1)


# ---------------------------------------------------------------------------
# troubled-cell gate: seeded network parameters and synthetic samples
# ---------------------------------------------------------------------------
GATE_IN, GATE_H = 24, 32
GATE_NPARAM = GATE_H * GATE_IN + GATE_H + GATE_H * GATE_H + GATE_H + GATE_H + 1 + 2 * GATE_IN


def gate_init(seed: int = 2312) -> np.ndarray:
    """Float32 parameter vector W1[32][24], b1, W2[32][32], b2, w3, b3, mean[24],
    inv_std[24]: He-scaled normal weights, zero biases, mean 0, inv_std 1."""
    z = normal01(seed, GATE_H * GATE_IN + GATE_H * GATE_H + GATE_H)
    P = np.zeros(GATE_NPARAM, dtype=np.float64)
    o = 0
    P[o:o + GATE_H * GATE_IN] = z[:GATE_H * GATE_IN] * math.sqrt(2.0 / GATE_IN)
    o += GATE_H * GATE_IN + GATE_H
    P[o:o + GATE_H * GATE_H] = z[GATE_H * GATE_IN:GATE_H * (GATE_IN + GATE_H)] * math.sqrt(2.0 / GATE_H)
    o += GATE_H * GATE_H + GATE_H
    P[o:o + GATE_H] = z[GATE_H * (GATE_IN + GATE_H):] * math.sqrt(1.0 / GATE_H)
    o += GATE_H + 1
    P[o + GATE_IN:] = 1.0
    return P.astype(np.float32)


def gate_samples(n: int, seed: int = 2313, scale: float = 0.4):
    """n synthetic gate inputs (float32 [n][24], normal with the given scale,
    clipped to [-1, 1] like the normalised features) and Bernoulli(0.3) labels."""
    X = np.clip(scale * normal01(seed, n * GATE_IN).reshape(n, GATE_IN), -1.0, 1.0).astype(np.float32)
    y = (uniform01(seed + 1, n) < 0.3).astype(np.float32)
    return X, y
