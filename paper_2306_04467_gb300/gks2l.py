"""Thin Python binding of the gks2l C ABI (include/gks2l.h).

Argument marshalling only: every step of the scheme runs in the CUDA library.
Device memory (the workspace) and the stream come from PyTorch. There is no
CPU fallback: importing works without a GPU, but creating a solver raises if
the compiled library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgks2l.so")

GKS2L_FP64 = 0
GKS2L_FP32 = 1
GKS2L_INDICATOR_OFF = 0
GKS2L_INDICATOR_MLP = 1
GKS2L_BC_INTERIOR = 0
GKS2L_BC_WALL = 1
GKS2L_BC_PERIODIC = 2
GKS2L_MLP_NPARAM = 1937
GKS2L_MLP_NTRAIN = 1889
GKS2L_OK = 0
GKS2L_EINVAL = -1
GKS2L_EMESH = -2
GKS2L_ECUDA = -3
GKS2L_ESTATE = -4
GKS2L_ENEGDEPTH = -5
GKS2L_ENONFINITE = -6
GKS2L_ESPACE = -7
GKS2L_ENOTIMPL = -8
GKS2L_ETOOBIG = -9
GKS2L_ETIMEOUT = -10
GKS2L_LAUNCH_SHAPES = 5
GKS2L_GATE_KERNELS = 4
GKS2L_GATE_VARIANTS = 16

# every entry point the header declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


class gks2l_mesh(ctypes.Structure):
    _fields_ = [("n_vert", ctypes.c_int32), ("xy", _P), ("n_tri", ctypes.c_int32), ("tri", _P),
                ("tri_bc", _P), ("period", ctypes.c_double * 2)]


class gks2l_params(ctypes.Structure):
    _fields_ = [("g", _D), ("chi", _D), ("cfl", _D), ("eps", _D), ("eps_num", _D),
                ("weno_gamma_hi", _D), ("weno_eps", _D), ("precision", ctypes.c_int32),
                ("indicator", ctypes.c_int32), ("indicator_threshold", ctypes.c_float),
                ("staging_poll_limit", ctypes.c_int32), ("positivity_floor", _D)]


class gks2l_stats_t(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 2), ("t", _D), ("dt_last", _D), ("stages_done", ctypes.c_int64),
                ("status", ctypes.c_int32), ("n_instances", ctypes.c_int32), ("smooth_fraction", _D)]


SIGNATURES = {
    "gks2l_default_params": (_I, [ctypes.POINTER(gks2l_params)]),
    "gks2l_create": (_I, [ctypes.POINTER(gks2l_mesh), ctypes.POINTER(gks2l_params), ctypes.POINTER(_P)]),
    "gks2l_create_ensemble": (_I, [ctypes.c_int32, ctypes.POINTER(gks2l_mesh), ctypes.POINTER(gks2l_params),
                                   ctypes.POINTER(_P)]),
    "gks2l_workspace_bytes": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "gks2l_bind": (_I, [_P, _P, ctypes.c_size_t, _P]),
    "gks2l_set_bathymetry": (_I, [_P, _P]),
    "gks2l_set_state": (_I, [_P, _P, _P]),
    "gks2l_set_state_device": (_I, [_P, _P, _P]),
    "gks2l_advance": (_I, [_P, ctypes.c_int32, _D, ctypes.POINTER(_D)]),
    "gks2l_get_state": (_I, [_P, _P, _P]),
    "gks2l_get_state_device": (_I, [_P, _P, _P]),
    "gks2l_run_items": (_I, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P]),
    "gks2l_stats": (_I, [_P, ctypes.POINTER(gks2l_stats_t)]),
    "gks2l_profile_kernels": (_I, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double * 6)]),
    "gks2l_set_launch_shapes": (_I, [_P, ctypes.POINTER(ctypes.c_int32 * 4)]),
    "gks2l_autotune": (_I, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32 * 4)]),
    "gks2l_alu_peaks": (_I, [_P, ctypes.POINTER(ctypes.c_double * 2)]),
    "gks2l_set_mlp": (_I, [_P, _P, ctypes.c_size_t]),
    "gks2l_harvest": (_I, [_P, ctypes.c_float, _P, _P, _P]),
    "gks2l_mlp_grad": (_I, [_P, _P, ctypes.c_int32, _P, ctypes.c_float, _P, _P, _P]),
    "gks2l_mlp_adam": (_I, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P]),
    "gks2l_mlp_forward": (_I, [_P, ctypes.c_int32, _P, _P, _P]),
    "gks2l_cfl_mass_noalloc": (_I, [ctypes.c_int32, _P, _P, _P, _D, _D, _P, _P]),
    "gks2l_error_string": (ctypes.c_char_p, [_I]),
    "gks2l_destroy": (None, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("gks2l CUDA library not built (%s): run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GKSError(RuntimeError):
    """A gks2l call returned a GKS2L_E* code (kept in .code)."""

    def __init__(self, msg, code=0):
        super().__init__(msg)
        self.code = code


def _check(rc, what):
    if rc != 0:
        msg = load().gks2l_error_string(rc).decode()
        raise GKSError("%s failed: %s (%d)" % (what, msg, rc), rc)


def _np_ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


def default_params(**kw) -> gks2l_params:
    p = gks2l_params()
    _check(load().gks2l_default_params(ctypes.byref(p)), "gks2l_default_params")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class _MeshArrays:
    """Keeps the numpy arrays a gks2l_mesh points to alive."""

    def __init__(self, mesh):
        self.xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        self.tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self.bc = np.ascontiguousarray(mesh.tri_bc, dtype=np.int8)
        self.s = gks2l_mesh(mesh.n_vert, _np_ptr(self.xy), mesh.n_tri, _np_ptr(self.tri), _np_ptr(self.bc),
                            (ctypes.c_double * 2)(float(mesh.period[0]), float(mesh.period[1])))


class Solver:
    """One bound gks2l context on the current CUDA device.

    meshes: one inputs.Mesh or a list of them (an ensemble).
    """

    def __init__(self, meshes, params: gks2l_params, b_vert=None, device="cuda", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("gks2l needs a CUDA device; no CPU fallback exists")
        L = load()
        self.torch = torch
        if not isinstance(meshes, (list, tuple)):
            meshes = [meshes]
        self._arrs = [_MeshArrays(m) for m in meshes]
        arr = (gks2l_mesh * len(meshes))(*[a.s for a in self._arrs])
        self.n_tri = sum(m.n_tri for m in meshes)
        self.n_vert = sum(m.n_vert for m in meshes)
        self.params = params
        h = _P()
        if len(meshes) == 1:
            rc = L.gks2l_create(arr, ctypes.byref(params), ctypes.byref(h))
        else:
            rc = L.gks2l_create_ensemble(len(meshes), arr, ctypes.byref(params), ctypes.byref(h))
        _check(rc, "gks2l_create")
        self._h = h
        self._gate_variant = 0
        nbytes = ctypes.c_size_t(0)
        _check(L.gks2l_workspace_bytes(h, ctypes.byref(nbytes)), "gks2l_workspace_bytes")
        self.device = torch.device(device)
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check(L.gks2l_bind(h, _P(self.workspace.data_ptr()), int(nbytes.value), _P(self.stream.cuda_stream)),
               "gks2l_bind")
        if b_vert is not None:
            self.set_bathymetry(b_vert)

    @property
    def workspace_bytes(self):
        return self.workspace.numel()

    def set_bathymetry(self, b_vert):
        b = np.ascontiguousarray(b_vert, dtype=np.float64)
        assert b.size == self.n_vert
        self._b = b
        _check(load().gks2l_set_bathymetry(self._h, _np_ptr(b)), "gks2l_set_bathymetry")

    def set_state(self, avg, grad=None):
        """Host arrays (numpy, variable-major, caller order)."""
        a = np.ascontiguousarray(avg, dtype=np.float64)
        g = None if grad is None else np.ascontiguousarray(grad, dtype=np.float64)
        assert a.size == 6 * self.n_tri and (g is None or g.size == 12 * self.n_tri)
        _check(load().gks2l_set_state(self._h, _np_ptr(a), _np_ptr(g)), "gks2l_set_state")

    def set_state_host_ptr(self, avg_ptr: int, grad_ptr: int):
        """Host pointers (e.g. pinned torch tensors)."""
        _check(load().gks2l_set_state(self._h, _P(avg_ptr), _P(grad_ptr)), "gks2l_set_state")

    def set_state_device(self, avg, grad=None):
        """Device tensors (float64, contiguous, caller order)."""
        _check(load().gks2l_set_state_device(self._h, _P(avg.data_ptr()),
                                             _P(grad.data_ptr()) if grad is not None else None),
               "gks2l_set_state_device")

    def advance(self, n_stages, t_end=0.0, sync=True):
        t = ctypes.c_double(0)
        rc = load().gks2l_advance(self._h, int(n_stages), float(t_end), ctypes.byref(t) if sync else None)
        _check(rc, "gks2l_advance")
        return t.value if sync else None

    def get_state(self):
        a = np.zeros((6, self.n_tri))
        g = np.zeros((6, 2, self.n_tri))
        _check(load().gks2l_get_state(self._h, _np_ptr(a), _np_ptr(g)), "gks2l_get_state")
        return a, g

    def get_state_host_ptr(self, avg_ptr: int, grad_ptr: int):
        _check(load().gks2l_get_state(self._h, _P(avg_ptr), _P(grad_ptr)), "gks2l_get_state")

    def get_state_device(self, avg, grad=None):
        _check(load().gks2l_get_state_device(self._h, _P(avg.data_ptr()),
                                             _P(grad.data_ptr()) if grad is not None else None),
               "gks2l_get_state_device")

    def run_items(self, inputs, outputs, n_stages):
        """Pipelined host I/O (gks2l_run_items): inputs[i] = (avg, grad) and
        outputs[i] = (avg, grad) host arrays of item i, each a numpy float64
        array (C-contiguous, the set_state / get_state layout), a CPU torch
        tensor (pinned for overlap) or None for grad. Every item is set,
        advanced n_stages stages and read back; the copies of neighbouring
        items overlap the computation."""
        n = len(inputs)
        if len(outputs) != n:
            raise ValueError("inputs and outputs differ in length")

        def ptr(x, writable):
            if x is None:
                return None
            if isinstance(x, np.ndarray):
                if x.dtype != np.float64 or not x.flags.c_contiguous or (writable and not x.flags.writeable):
                    raise ValueError("host arrays must be C-contiguous float64" + (" and writable" if writable else ""))
                return x.ctypes.data
            if x.is_cuda or x.dtype != self.torch.float64 or not x.is_contiguous():
                raise ValueError("tensors must be contiguous float64 CPU tensors (pinned for overlap)")
            return x.data_ptr()

        arr = ctypes.c_void_p * max(n, 1)
        ia, ig = arr(*[ptr(a, False) for a, _ in inputs]), arr(*[ptr(g, False) for _, g in inputs])
        oa, og = arr(*[ptr(a, True) for a, _ in outputs]), arr(*[ptr(g, True) for _, g in outputs])
        _check(load().gks2l_run_items(self._h, n, int(n_stages), ia, ig, oa, og), "gks2l_run_items")

    def stats(self) -> dict:
        s = gks2l_stats_t()
        _check(load().gks2l_stats(self._h, ctypes.byref(s)), "gks2l_stats")
        return {"mass": (s.mass[0], s.mass[1]), "t": s.t, "dt": s.dt_last, "stages": s.stages_done,
                "status": s.status, "n_instances": s.n_instances, "smooth_fraction": s.smooth_fraction}

    def profile_kernels(self, n_steps):
        """Mean ms per launch of recon, iface, edge, update, step_begin, gate."""
        ms = (ctypes.c_double * 6)()
        _check(load().gks2l_profile_kernels(self._h, int(n_steps), ctypes.byref(ms)), "gks2l_profile_kernels")
        return {"recon": ms[0], "iface": ms[1], "edge": ms[2], "update": ms[3], "step_begin": ms[4], "gate": ms[5]}

    def set_launch_shapes(self, shapes):
        """Launch shapes (0..4) of the interface, edge and update kernels and,
        as a fourth entry, the gate variant (0..15: kernel = v % 4, placement
        = v // 4 % 2, edge path = v // 8; kept at the current choice when
        only three are given)."""
        shapes = [int(x) for x in shapes]
        if len(shapes) == 3:
            shapes.append(self._gate_variant)
        b = (ctypes.c_int32 * 4)(*shapes)
        _check(load().gks2l_set_launch_shapes(self._h, ctypes.byref(b)), "gks2l_set_launch_shapes")
        self._gate_variant = shapes[3]

    def autotune(self, n_steps=2):
        """Time each launch shape for n_steps steps (they advance the state);
        keep the fastest per kernel (and, with the gate on, the faster gate
        kernel by whole steps) and return the four choices."""
        b = (ctypes.c_int32 * 4)()
        _check(load().gks2l_autotune(self._h, int(n_steps), ctypes.byref(b)), "gks2l_autotune")
        self._gate_variant = b[3]
        return list(b)

    def alu_peaks(self):
        """Measured FP32 and FP64 FMA throughput of the device, TFLOP/s."""
        t = (ctypes.c_double * 2)()
        _check(load().gks2l_alu_peaks(self._h, ctypes.byref(t)), "gks2l_alu_peaks")
        return {"fp32": t[0], "fp64": t[1]}

    def set_mlp(self, params_f32: np.ndarray):
        p = np.ascontiguousarray(params_f32, dtype=np.float32)
        _check(load().gks2l_set_mlp(self._h, _np_ptr(p), p.size), "gks2l_set_mlp")

    def harvest(self, tol, features=None, labels=None, logits=None):
        """Gate training data of the current state (device tensors, caller's
        cell order): features [n_tri, 24], labels [n_tri], optionally the fused
        gate's logits [n_tri]. Allocates what is not given; returns the three."""
        n, torch = self.n_tri, self.torch
        if features is None:
            features = torch.empty((n, 24), dtype=torch.float32, device=self.device)
        if labels is None:
            labels = torch.empty(n, dtype=torch.float32, device=self.device)
        _check(load().gks2l_harvest(self._h, float(tol), _P(features.data_ptr()), _P(labels.data_ptr()),
                                    _P(logits.data_ptr()) if logits is not None else None), "gks2l_harvest")
        return features, labels, logits

    def close(self):
        if getattr(self, "_h", None):
            load().gks2l_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cfl_mass_noalloc(avg, area, dX, g, cfl, out, stream=None):
    """gks2l_cfl_mass_noalloc on device tensors (float64, same cell order):
    writes (dt, mass of layer 1, mass of layer 2, number of unusable cells)
    into `out` (4 doubles)."""
    n = area.numel()
    s = _P(stream.cuda_stream) if stream is not None else None
    _check(load().gks2l_cfl_mass_noalloc(n, _P(avg.data_ptr()), _P(area.data_ptr()), _P(dX.data_ptr()),
                                         float(g), float(cfl), _P(out.data_ptr()), s), "gks2l_cfl_mass_noalloc")


def _sp(stream):
    return _P(stream.cuda_stream) if stream is not None else None


def mlp_grad(X, y, params, pos_weight, grads, loss, stream=None):
    """Summed loss gradient of the gate network on device tensors."""
    _check(load().gks2l_mlp_grad(_P(X.data_ptr()), _P(y.data_ptr()), int(y.numel()), _P(params.data_ptr()),
                                 float(pos_weight), _P(grads.data_ptr()), _P(loss.data_ptr()), _sp(stream)),
           "gks2l_mlp_grad")


def mlp_adam(params, grads, m, v, step, lr, scale, stream=None):
    _check(load().gks2l_mlp_adam(_P(params.data_ptr()), _P(grads.data_ptr()), _P(m.data_ptr()), _P(v.data_ptr()),
                                 int(step), float(lr), float(scale), _sp(stream)), "gks2l_mlp_adam")


def mlp_forward(X, params, logits, stream=None):
    _check(load().gks2l_mlp_forward(_P(X.data_ptr()), int(logits.numel()), _P(params.data_ptr()),
                                    _P(logits.data_ptr()), _sp(stream)), "gks2l_mlp_forward")


def problem_solver(prob, precision=GKS2L_FP64, **kw):
    """Solver for an inputs.Problem with its parameters and initial state."""
    p = default_params(g=prob.g, chi=prob.chi, cfl=prob.cfl, eps=prob.eps, eps_num=prob.eps_num,
                       precision=precision, **kw)
    s = Solver(prob.mesh, p, prob.b_vert)
    s.set_state(prob.avg, prob.grad)
    return s
