"""Host-side checks of the C ABI that need no GPU: the library loads, it
exports every function include/lbib.h declares, and parameter / workspace
validation returns the documented codes before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import lbib_inputs as li

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1503_06726_gb300 import build
    build.build()
    from paper_1503_06726_gb300 import lbib
    return lbib


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbib_\w+)\s*\(", txt, re.M))
    return names


def test_exports_every_declared_symbol(L):
    lib = L.load()
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(L.EXPORTS)


def test_workspace_size_and_param_validation(L):
    w = li.config2()
    p = L.make_params(w.params, L.LBIB_FP32)
    n = L.lbib_workspace_size(p, w.tissue.n_vertices, w.tissue.n_cells)
    # populations dominate: 2 buffers x (9 + 5*2) planes x 4 bytes
    assert n >= 2 * 19 * 1024 * 1024 * 4
    for field, bad in (("tau", 0.5), ("nx", 4), ("n_species", 5), ("bc_y", 3),
                       ("precision", 7), ("rho0", 0.0)):
        q = L.make_params(w.params, L.LBIB_FP32)
        setattr(q, field, bad)
        with pytest.raises(L.LbibError) as e:
            L.lbib_workspace_size(q, 10, 1)
        assert e.value.code == L.LBIB_E_PARAM
    q = L.make_params(w.params, L.LBIB_FP32)
    q.D[1] = 0.0
    with pytest.raises(L.LbibError):
        L.lbib_workspace_size(q, 10, 1)


def test_create_rejects_bad_workspace_without_touching_device(L):
    w = li.config1()
    p = L.make_params(w.params, L.LBIB_FP64)
    with pytest.raises(L.LbibError) as e:
        L.lbib_create(p, 64, 1, 0, 1 << 20, 0)
    assert e.value.code == L.LBIB_E_WORKSPACE
    with pytest.raises(L.LbibError) as e:
        L.lbib_create(p, 64, 1, 0x1000010, 1 << 30, 0)   # misaligned
    assert e.value.code == L.LBIB_E_WORKSPACE
    need = L.lbib_workspace_size(p, 64, 1)
    with pytest.raises(L.LbibError) as e:
        L.lbib_create(p, 64, 1, 0x1000000, need - 256, 0)
    assert e.value.code == L.LBIB_E_WORKSPACE
    assert "too small" in L.lbib_last_error(None)


def test_status_strings(L):
    assert L.lbib_status_string(0) == "LBIB_OK"
    assert L.lbib_status_string(-5) == "LBIB_E_TIMEOUT"
