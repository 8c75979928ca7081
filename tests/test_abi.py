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


def test_option_validation_on_the_host(L):
    """The options of the rows beyond the plain step are checked by the host
    before any device work: reaction models, confined species, junctions,
    mass sources, pressure and node sources (lbib_workspace_size runs the
    same checks as lbib_create)."""
    w = li.config2(nx=96, ny=80, n_cells_side=3)
    bad = (("reaction", 7), ("noflux_mask", 1 << 3),
           ("junction_period", -1), ("mass_sources", 2), ("pressure_nodes", 2),
           ("node_sources", 2))
    for field, value in bad:
        q = L.make_params(w.params, L.LBIB_FP32)
        setattr(q, field, value)
        with pytest.raises(L.LbibError) as e:
            L.lbib_workspace_size(q, 10, 1)
        assert e.value.code == L.LBIB_E_PARAM, field
    # junctions: l_max must leave room for the 3x3 bin search
    q = L.make_params(w.params, L.LBIB_FP32)
    q.junction_period, q.junction_lmax, q.junction_k = 5, 40.0, 0.01
    with pytest.raises(L.LbibError):
        L.lbib_workspace_size(q, 10, 1)
    # pressure nodes need a positive density
    q = L.make_params(w.params, L.LBIB_FP32)
    q.pressure_nodes, q.pressure_rho = 1, 0.0
    with pytest.raises(L.LbibError):
        L.lbib_workspace_size(q, 10, 1)
    # valid options enlarge the workspace by their planes
    base = L.lbib_workspace_size(L.make_params(w.params, L.LBIB_FP32), 900, 9)
    q = L.make_params(w.params, L.LBIB_FP32)
    q.junction_period, q.junction_lmax, q.junction_k = 5, 8.0, 0.01
    q.mass_sources, q.pressure_nodes, q.pressure_rho, q.node_sources = 1, 1, 1.0, 1
    assert L.lbib_workspace_size(q, 900, 9) > base


def test_binding_refuses_options_without_a_cuda_path(L):
    w = li.config2(nx=96, ny=80, n_cells_side=3)
    w.params.mass_beta = 1e-3
    with pytest.raises(ValueError):
        L.make_params(w.params, L.LBIB_FP32)
    w.params.mass_beta, w.params.noflux, w.params.noflux_dynamic = 0.0, 1, 1
    with pytest.raises(ValueError):
        L.make_params(w.params, L.LBIB_FP32)


def test_nvtx_ranges_are_built_in(L):
    """The host calls that enqueue device work open named NVTX ranges (a
    profiler's timeline shows them around their launches); their names are in
    the library."""
    from paper_1503_06726_gb300 import build
    blob = open(build.LIB, "rb").read()
    for name in (b"lbib_step", b"lbib_advance", b"lbib.lattice_update", b"lbib.ib_cells",
                 b"lbib_get_fields", b"lbib_get_sums", b"lbib_ensemble_step",
                 b"lbib_steady_solve", b"lbib_nop_train_step", b"nn.conv3x3",
                 b"nn.conv3x3_wgrad"):
        assert name + b"\x00" in blob, name
