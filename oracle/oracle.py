"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this
module. It shares no code with the CUDA path; both take their inputs from the
seeded generators in paper_2306_04467_gb300.inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

# default scheme constants: collision time (Sec. 4) and the WENO reading
EPS = 0.05
EPS_NUM = 5.0
GAMMA_HI = 0.85
WENO_EPS = 1.0


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.c_double
        p = ctypes.c_void_p
        i = ctypes.c_int
        _lib.orc_create.restype = p
        _lib.orc_create.argtypes = [i, p, i, p, p, d, d, p, d, d, d, d, d, d, d, ctypes.POINTER(i)]
        _lib.orc_destroy.argtypes = [p]
        _lib.orc_num_edges.argtypes = [p]
        _lib.orc_set_state.argtypes = [p, p, p]
        _lib.orc_get_state.argtypes = [p, p, p]
        _lib.orc_advance.argtypes = [p, i, d, ctypes.POINTER(d)]
        _lib.orc_last_dt.argtypes = [p]
        _lib.orc_last_dt.restype = d
        _lib.orc_time.argtypes = [p]
        _lib.orc_time.restype = d
        _lib.orc_mass.argtypes = [p, p]
        _lib.orc_cell_geometry.argtypes = [p, p, p, p]
        _lib.orc_reconstruct.argtypes = [p]
        _lib.orc_set_positivity.argtypes = [p, d]
        _lib.orc_positivity_scale.argtypes = [p]
        _lib.orc_eval.argtypes = [p, i, d, d, p, p]
        _lib.orc_omega.argtypes = [p, p]
        _lib.orc_weight_departure.argtypes = [p, p]
        _lib.orc_set_linear_mask.argtypes = [p, p]
        _lib.orc_gate_features.argtypes = [p, p]
        _lib.orc_stencil_size.argtypes = [p, i]
        _lib.orc_edge_points.argtypes = [p, p, p]
        _lib.orc_blend_levels.argtypes = [p, p]
        _lib.orc_plane_gradients.argtypes = [p, p]
        _lib.orc_gauss_gradient.argtypes = [p, p, p]
        _lib.orc_edge_outputs.argtypes = [p, p, p, p, p]
        _lib.orc_raw_moments.argtypes = [d, d, i, i, p]
        _lib.orc_time_integrals.argtypes = [d, d, p]
        _lib.orc_gks_point.argtypes = [p, p, d, d, d, p, p]
        _lib.orc_s2o4.argtypes = [i, d, d, d, d, d]
        _lib.orc_s2o4.restype = d
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One oracle instance on a mesh with vertex bathymetry and parameters."""

    def __init__(self, mesh, b_vert=None, g=9.81, chi=0.98, cfl=0.5, eps=EPS, eps_num=EPS_NUM,
                 gamma_hi=GAMMA_HI, weno_eps=WENO_EPS):
        L = lib()
        self.mesh = mesh
        self.nt = mesh.n_tri
        self._xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        self._tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self._bc = np.ascontiguousarray(mesh.tri_bc, dtype=np.int8)
        bv = np.zeros(mesh.n_vert) if b_vert is None else b_vert
        self._bv = np.ascontiguousarray(bv, dtype=np.float64)
        st = ctypes.c_int(0)
        self._h = L.orc_create(mesh.n_vert, _ptr(self._xy), mesh.n_tri, _ptr(self._tri), _ptr(self._bc),
                               float(mesh.period[0]), float(mesh.period[1]), _ptr(self._bv),
                               g, chi, cfl, eps, eps_num, gamma_hi, weno_eps, ctypes.byref(st))
        if st.value != 0:
            L.orc_destroy(self._h)
            self._h = None
            raise RuntimeError("oracle mesh set-up failed with status %d" % st.value)
        self.ne = L.orc_num_edges(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    @classmethod
    def from_problem(cls, prob, **kw):
        o = cls(prob.mesh, prob.b_vert, g=prob.g, chi=prob.chi, cfl=prob.cfl, eps=prob.eps,
                eps_num=prob.eps_num, **kw)
        o.set_state(prob.avg, prob.grad)
        return o

    def set_state(self, avg, grad):
        a = np.ascontiguousarray(avg, dtype=np.float64).reshape(6, self.nt)
        g = np.ascontiguousarray(grad, dtype=np.float64).reshape(6, 2, self.nt)
        lib().orc_set_state(self._h, _ptr(a), _ptr(g))

    def get_state(self):
        a = np.zeros((6, self.nt))
        g = np.zeros((6, 2, self.nt))
        lib().orc_get_state(self._h, _ptr(a), _ptr(g))
        return a, g

    def advance(self, n_stages, t_end=0.0):
        t = ctypes.c_double(0)
        st = lib().orc_advance(self._h, int(n_stages), float(t_end), ctypes.byref(t))
        if st != 0:
            why = {-10: "the CFL step is not a positive finite number (a non-physical state)",
                   -11: "a non-finite interface state appeared in the stage"}.get(st, "unknown")
            raise RuntimeError("oracle advance failed with status %d: %s" % (st, why))
        return t.value

    @property
    def t(self):
        return lib().orc_time(self._h)

    @property
    def dt(self):
        return lib().orc_last_dt(self._h)

    def mass(self):
        m = np.zeros(2)
        lib().orc_mass(self._h, _ptr(m))
        return m

    def geometry(self):
        a, x, y = np.zeros(self.nt), np.zeros(self.nt), np.zeros(self.nt)
        lib().orc_cell_geometry(self._h, _ptr(a), _ptr(x), _ptr(y))
        return a, x, y

    def reconstruct(self):
        lib().orc_reconstruct(self._h)

    def eval(self, c, x, y):
        v = np.zeros(6)
        g = np.zeros(12)
        lib().orc_eval(self._h, int(c), float(x), float(y), _ptr(v), _ptr(g))
        return v, g.reshape(6, 2)

    def omega(self):
        om = np.zeros(self.nt * 6)
        lib().orc_omega(self._h, _ptr(om))
        return om.reshape(self.nt, 6)

    def weight_departure(self):
        """max_k |omega_k / gamma_k - 1| per (cell, variable) of the last reconstruction."""
        out = np.zeros(self.nt * 6)
        lib().orc_weight_departure(self._h, _ptr(out))
        return out.reshape(self.nt, 6)

    def set_positivity(self, floor_fraction):
        """The positivity option (not in the paper; 0 = off, the default):
        point depths held to floor_fraction of the cell's average depth by
        scaling the layer's depth and discharge polynomials, point velocities
        held within the edge's two cells' average velocities."""
        lib().orc_set_positivity(self._h, float(floor_fraction))

    def positivity_scale(self):
        """Apply the option's polynomial scaling to the current
        reconstruction (after reconstruct(); the velocity bound is not
        involved)."""
        lib().orc_positivity_scale(self._h)

    def set_linear_mask(self, mask):
        """Cells with mask = 1 take the linear weights from now on (None: none)."""
        if mask is None:
            lib().orc_set_linear_mask(self._h, None)
            return
        self._mask = np.ascontiguousarray(mask, dtype=np.uint8)
        assert self._mask.shape == (self.nt,)
        lib().orc_set_linear_mask(self._h, _ptr(self._mask))

    def gate_features(self):
        """The 24 troubled-cell gate inputs of every cell at the current state."""
        X = np.zeros(self.nt * 24)
        lib().orc_gate_features(self._h, _ptr(X))
        return X.reshape(self.nt, 24)

    def stencil_size(self, c):
        return lib().orc_stencil_size(self._h, int(c))

    def edge_points(self):
        xq = np.zeros((self.ne, 2, 2))
        lr = np.zeros((self.ne, 2), dtype=np.int32)
        lib().orc_edge_points(self._h, _ptr(xq), _ptr(lr))
        return xq, lr

    def blend_levels(self):
        """Edge-centre blended levels of the last stage (Sec. 2.3): [ne, 2] =
        (lower-layer depth h1-hat, upper-layer h2-hat)."""
        hc = np.zeros(2 * self.ne)
        lib().orc_blend_levels(self._h, _ptr(hc))
        return hc.reshape(self.ne, 2)

    def plane_gradients(self):
        """Per cell, the gradients of the planes through its three edge-centre
        blended levels of the last stage (Sec. 2.3): [nt, 2, 2] = (h1-hat,
        h2-hat) x (d/dx, d/dy)."""
        pg = np.zeros(4 * self.nt)
        lib().orc_plane_gradients(self._h, _ptr(pg))
        return pg.reshape(self.nt, 2, 2)

    def gauss_gradient(self, point_values):
        pv = np.ascontiguousarray(point_values, dtype=np.float64).reshape(self.ne, 2)
        g = np.zeros((self.nt, 2))
        lib().orc_gauss_gradient(self._h, _ptr(pv), _ptr(g))
        return g

    def edge_outputs(self):
        out = [np.zeros((self.ne, 2, 6)) for _ in range(4)]
        lib().orc_edge_outputs(self._h, *[_ptr(a) for a in out])
        return out


def raw_moments(U, lam, half, n):
    mu = np.zeros(n + 1)
    lib().orc_raw_moments(float(U), float(lam), int(half), int(n), _ptr(mu))
    return mu


def time_integrals(tau, delta):
    q = np.zeros(5)
    lib().orc_time_integrals(float(tau), float(delta), _ptr(q))
    return q


def gks_point(left, right, g, tau, delta):
    """left/right: (h, U, V, dn[3], dt[3], phin, phit) in the local frame.
    Returns the time-integrated moments (W_int[3], F_int[3]) over [0, delta]."""
    l = np.ascontiguousarray(left, dtype=np.float64)
    r = np.ascontiguousarray(right, dtype=np.float64)
    W = np.zeros(3)
    F = np.zeros(3)
    lib().orc_gks_point(_ptr(l), _ptr(r), float(g), float(tau), float(delta), _ptr(W), _ptr(F))
    return W, F


def s2o4(stage, Wn, Ln, Ltn, Lt_half, dt):
    return lib().orc_s2o4(int(stage), Wn, Ln, Ltn, Lt_half, dt)
