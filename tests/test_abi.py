"""The C ABI library builds, loads without a GPU and exports every entry point
the public header declares; the binding covers each of them."""
import os
import re

import pytest

from paper_2306_04467_gb300 import build as B
from paper_2306_04467_gb300 import gks2l

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gks2l.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gks2l_[a-z_]+)\s*\(", text)))


def test_library_builds_and_exports_all_declared_symbols():
    path = B.build()
    import ctypes
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert set(declared_functions()) == set(gks2l.SIGNATURES)


def test_host_only_calls_work_without_gpu():
    lib = gks2l.load()
    p = gks2l.default_params()
    assert p.g == 9.81 and p.cfl == 0.5 and p.eps == 0.05 and p.eps_num == 5.0
    assert lib.gks2l_error_string(0) == b"ok"


def test_workspace_size_is_known_on_the_host():
    """gks2l_create and gks2l_workspace_bytes touch no GPU: a caller sizes the
    workspace before any device memory exists, for one mesh and for an
    ensemble, in either precision (the FP32 form needs less)."""
    import ctypes
    from paper_2306_04467_gb300 import inputs
    lib = gks2l.load()
    meshes = [inputs.smooth_periodic(16).mesh, inputs.lake_at_rest(24).mesh, inputs.smooth_periodic(8).mesh]
    keep = [gks2l._MeshArrays(m) for m in meshes]
    sizes = {}
    for prec in (gks2l.GKS2L_FP64, gks2l.GKS2L_FP32):
        par = gks2l.default_params(precision=prec)
        for n in (1, 3):
            arr = (gks2l.gks2l_mesh * n)(*[k.s for k in keep[:n]])
            h = gks2l._P()
            if n == 1:
                rc = lib.gks2l_create(arr, ctypes.byref(par), ctypes.byref(h))
            else:
                rc = lib.gks2l_create_ensemble(n, arr, ctypes.byref(par), ctypes.byref(h))
            assert rc == 0
            nb = ctypes.c_size_t(0)
            assert lib.gks2l_workspace_bytes(h, ctypes.byref(nb)) == 0
            n_tri = sum(m.n_tri for m in meshes[:n])
            assert 1000 * n_tri < nb.value < 8000 * n_tri
            sizes[prec, n] = nb.value
            lib.gks2l_destroy(h)
    for n in (1, 3):
        assert sizes[gks2l.GKS2L_FP32, n] < sizes[gks2l.GKS2L_FP64, n]
