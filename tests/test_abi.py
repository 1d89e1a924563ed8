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
