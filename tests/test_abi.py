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


def test_binding_constants_match_the_header():
    """Every GKS2L_ constant the header defines has the same value in the
    binding, and the parameter struct has the header's fields in order."""
    text = open(HEADER).read()
    defs = dict(re.findall(r"#define (GKS2L_[A-Z0-9_]+)\s+(-?\d+)\s", text))
    assert len(defs) >= 20
    for name, val in defs.items():
        assert getattr(gks2l, name) == int(val), name
    body = re.search(r"typedef struct \{([^}]*)\} gks2l_params;", text).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)\s*[,;]", body)
    assert fields == [f for f, _ in gks2l.gks2l_params._fields_]


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


def _create(xy, tri, bc=None, period=(0.0, 0.0), **par):
    """gks2l_create on host arrays (no GPU is touched); returns its code and
    destroys a context it made."""
    import ctypes
    import numpy as np
    lib = gks2l.load()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    bcp = None
    if bc is not None:
        bc = np.ascontiguousarray(bc, dtype=np.int8)
        bcp = bc.ctypes.data_as(gks2l._P)
    m = gks2l.gks2l_mesh(len(xy), xy.ctypes.data_as(gks2l._P), len(tri), tri.ctypes.data_as(gks2l._P), bcp,
                         (ctypes.c_double * 2)(*period))
    p = gks2l.default_params(**par)
    h = gks2l._P()
    rc = lib.gks2l_create(ctypes.byref(m), ctypes.byref(p), ctypes.byref(h))
    if rc == 0:
        lib.gks2l_destroy(h)
    return rc


def test_create_rejects_unusable_input_on_the_host():
    """Bad meshes and parameters come back as error codes from gks2l_create
    (never a crash): an empty mesh or a bad parameter is EINVAL; a vertex
    index out of range, a clockwise triangle, a periodic side without a
    partner or one whose partner is not its translate is EMESH. A square of
    two triangles with walls, or periodic with period 1, is accepted."""
    import numpy as np
    EINVAL, EMESH = -1, -2
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    ok = np.array([[0, 1, 2], [0, 2, 3]])
    assert _create(sq, ok) == 0
    assert _create(sq, ok[:0]) == EINVAL
    assert _create(sq, np.array([[0, 1, 7], [0, 2, 3]])) == EMESH
    assert _create(sq, np.array([[0, 2, 1], [0, 2, 3]])) == EMESH
    periodic = np.full((2, 3), 2, dtype=np.int8)
    assert _create(sq, ok, bc=periodic, period=(1.0, 1.0)) == 0
    assert _create(sq, ok, bc=periodic, period=(2.0, 2.0)) == EMESH      # no partners
    assert _create(sq, ok, bc=periodic, period=(0.5, 0.5)) == EMESH      # partners not translates
    for bad in (dict(g=0.0), dict(cfl=-1.0), dict(eps=0.0), dict(chi=0.0), dict(weno_gamma_hi=1.5),
                dict(precision=7)):
        assert _create(sq, ok, **bad) == EINVAL, bad
