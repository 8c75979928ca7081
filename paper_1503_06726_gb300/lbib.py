"""Thin Python binding of the C ABI in include/lbib.h (ctypes).

Argument marshalling only: every step of the coupled LB-IB path runs in the
CUDA library ``_build/liblbib.so``.  PyTorch provides the device workspace
(a uint8 CUDA tensor) and the stream; nothing here computes the method.
The functions keep the C names (``lbib_create``, ``lbib_step``, ...);
:class:`Simulation` bundles them for convenience.

Importing this module does not need a GPU, but loading the library does
need it to exist: there is no CPU fallback, and a missing library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbib.so")
# the checking build (bounds and alignment checks in the kernels), used when
# the environment sets LBIB_CHECK=1
LIB_CHECK_PATH = os.path.join(HERE, "_build_check", "liblbib_check.so")

LBIB_OK = 0
LBIB_E_PARAM = -1
LBIB_E_WORKSPACE = -2
LBIB_E_CELLS = -3
LBIB_E_NONFINITE = -4
LBIB_E_TIMEOUT = -5
LBIB_E_CUDA = -6
LBIB_E_STATE = -7
LBIB_E_CHECK = -8

LBIB_FP64, LBIB_FP32, LBIB_FP16 = 0, 1, 2
LBIB_GUO, LBIB_HE_PAPER = 0, 1
LBIB_REACT_LINEAR, LBIB_REACT_SCHNAKENBERG = 0, 1
LBIB_NOFLUX_CLOSURE, LBIB_NOFLUX_BOUNCEBACK = 0, 1
LBIB_ENS_PERSISTENT, LBIB_ENS_SPLIT, LBIB_ENS_SPLIT_WIDE = 0, 1, 2
LBIB_RHO, LBIB_U, LBIB_PHI, LBIB_X = 1, 2, 4, 8
LBIB_AREA, LBIB_ID, LBIB_FORCE, LBIB_VFORCE = 16, 32, 64, 128

PRECISIONS = {"fp64": LBIB_FP64, "fp32": LBIB_FP32, "fp16": LBIB_FP16}

# every symbol declared in include/lbib.h
EXPORTS = (
    "lbib_workspace_size", "lbib_create", "lbib_set_cells", "lbib_set_lattice_variant",
    "lbib_get_cells_async", "lbib_wait_readback",
    "lbib_set_domains", "lbib_set_mass_sources", "lbib_set_pressure_nodes",
    "lbib_set_node_sources",
    "lbib_set_cell_params",
    "lbib_set_species", "lbib_step", "lbib_advance", "lbib_get_sums", "lbib_step_profiled", "lbib_get_fields", "lbib_get_sizes", "lbib_state_size",
    "lbib_get_state", "lbib_set_state", "lbib_step_noalloc", "lbib_destroy", "lbib_last_error",
    "lbib_status_string", "lbib_label_cells", "lbib_steady_workspace_size", "lbib_steady_solve",
    "lbib_ensemble_workspace_size", "lbib_ensemble_create", "lbib_ensemble_tissue",
    "lbib_ensemble_step", "lbib_ensemble_status", "lbib_ensemble_config",
    "lbib_ensemble_schedule", "lbib_ensemble_tune",
    "lbib_ensemble_selftest_timeout", "lbib_ensemble_destroy", "lbib_ensemble_last_error",
    "lbib_nop_workspace_size", "lbib_nop_create", "lbib_nop_num_params", "lbib_nop_layers",
    "lbib_nop_set_params", "lbib_nop_get_params", "lbib_nop_get_grads", "lbib_nop_forward",
    "lbib_nop_train_step", "lbib_nop_destroy", "lbib_nop_last_error", "lbib_nn_conv3x3",
    "lbib_nn_conv3x3_wgrad", "lbib_nn_weight_copies", "lbib_nn_conv3x3_tc_supported",
    "lbib_nn_tile_weights_tc", "lbib_nn_conv3x3_tc", "lbib_nn_conv3x3_wgrad_tc_supported",
    "lbib_nn_conv3x3_wgrad_tc",
)


class LbibError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_status_name(code)} ({code}): {msg}")
        self.code = code


class lbib_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("n_species", ctypes.c_int32), ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("D", ctypes.c_double * 4), ("decay", ctypes.c_double * 4),
        ("react", (ctypes.c_double * 4) * 4), ("src_rate", ctypes.c_double * 4),
        ("forcing", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("fp16_scale", ctypes.c_double), ("fp16_scale_species", ctypes.c_double),
        ("tension", ctypes.c_double), ("body_force", ctypes.c_double * 2),
        ("reaction", ctypes.c_int32), ("noflux_mask", ctypes.c_int32),
        ("schnak", ctypes.c_double * 3),
        ("junction_k", ctypes.c_double), ("junction_l0", ctypes.c_double),
        ("junction_lmax", ctypes.c_double), ("junction_period", ctypes.c_int32),
        ("junction_pad", ctypes.c_int32),
        ("mass_sources", ctypes.c_int32), ("pressure_nodes", ctypes.c_int32),
        ("mass_alpha", ctypes.c_double), ("pressure_rho", ctypes.c_double),
        ("node_sources", ctypes.c_int32), ("noflux_scheme", ctypes.c_int32),
    ]


_lib = None


def load(path: str = None) -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built.  With
    LBIB_CHECK=1 in the environment the checking build is built if needed and
    loaded instead."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_PATH
        if os.environ.get("LBIB_CHECK") == "1":
            from . import build as _build
            path = _build.build(check=True)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
    P = ctypes.POINTER(lbib_params)
    sig = {
        "lbib_workspace_size": (ctypes.c_int, [P, i32, i32, ctypes.POINTER(u64)]),
        "lbib_create": (ctypes.c_int, [P, i32, i32, vp, u64, vp, ctypes.POINTER(vp)]),
        "lbib_set_cells": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "lbib_set_cell_params": (ctypes.c_int, [vp, vp, vp]),
        "lbib_set_lattice_variant": (ctypes.c_int, [vp, i32]),
        "lbib_get_cells_async": (ctypes.c_int, [vp, ctypes.c_uint32, vp, vp]),
        "lbib_wait_readback": (ctypes.c_int, [vp]),
        "lbib_set_domains": (ctypes.c_int, [vp, vp]),
        "lbib_set_mass_sources": (ctypes.c_int, [vp, vp, vp]),
        "lbib_set_pressure_nodes": (ctypes.c_int, [vp, vp]),
        "lbib_set_node_sources": (ctypes.c_int, [vp, vp]),
        "lbib_set_species": (ctypes.c_int, [vp, i32, vp]),
        "lbib_step": (ctypes.c_int, [vp, i32]),
        "lbib_advance": (ctypes.c_int, [vp, i32]),
        "lbib_get_sums": (ctypes.c_int, [vp, vp, vp, vp]),
        "lbib_step_profiled": (ctypes.c_int, [vp, i32, vp]),
        "lbib_get_fields": (ctypes.c_int, [vp, u32, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "lbib_get_sizes": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "lbib_state_size": (ctypes.c_int, [vp, ctypes.POINTER(u64)]),
        "lbib_get_state": (ctypes.c_int, [vp, vp, u64]),
        "lbib_set_state": (ctypes.c_int, [vp, vp, u64]),
        "lbib_step_noalloc": (ctypes.c_int, [P, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp]),
        "lbib_label_cells": (ctypes.c_int, [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp]),
        "lbib_steady_workspace_size": (ctypes.c_int, [i32, i32, i32, ctypes.POINTER(u64)]),
        "lbib_steady_solve": (ctypes.c_int, [i32, i32, i32, vp, vp, vp, vp, vp, ctypes.c_double,
                                             ctypes.c_int64, i32, vp, vp, vp, vp, vp, u64, vp]),
        "lbib_ensemble_workspace_size": (ctypes.c_int, [i32, P, vp, vp, ctypes.POINTER(u64)]),
        "lbib_ensemble_create": (ctypes.c_int, [i32, P, vp, vp, vp, u64, vp, ctypes.POINTER(vp)]),
        "lbib_ensemble_tissue": (vp, [vp, i32]),
        "lbib_ensemble_step": (ctypes.c_int, [vp, i32]),
        "lbib_ensemble_status": (ctypes.c_int, [vp]),
        "lbib_ensemble_config": (ctypes.c_int, [vp, i32, i32, vp, vp]),
        "lbib_ensemble_schedule": (ctypes.c_int, [vp, i32, vp]),
        "lbib_ensemble_tune": (ctypes.c_int, [vp, i32, vp, vp]),
        "lbib_ensemble_selftest_timeout": (ctypes.c_int, [vp, vp]),
        "lbib_ensemble_destroy": (None, [vp]),
        "lbib_ensemble_last_error": (ctypes.c_char_p, [vp]),
        "lbib_nop_workspace_size": (ctypes.c_int, [i32, i32, i32, ctypes.POINTER(u64)]),
        "lbib_nop_create": (ctypes.c_int, [i32, i32, i32, vp, u64, vp, ctypes.POINTER(vp)]),
        "lbib_nop_num_params": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "lbib_nop_layers": (ctypes.c_int, [vp, ctypes.POINTER(i32), vp]),
        "lbib_nop_set_params": (ctypes.c_int, [vp, vp, ctypes.c_int64]),
        "lbib_nop_get_params": (ctypes.c_int, [vp, vp, ctypes.c_int64]),
        "lbib_nop_get_grads": (ctypes.c_int, [vp, vp, ctypes.c_int64]),
        "lbib_nop_forward": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "lbib_nop_train_step": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp, vp, ctypes.c_double,
                                               i32, ctypes.POINTER(ctypes.c_double)]),
        "lbib_nop_destroy": (None, [vp]),
        "lbib_nop_last_error": (ctypes.c_char_p, [vp]),
        "lbib_nn_conv3x3": (ctypes.c_int, [i32] * 6 + [vp] * 5 + [i32, i32, vp]),
        "lbib_nn_conv3x3_wgrad": (ctypes.c_int, [i32] * 6 + [vp] * 5 + [vp]),
        "lbib_nn_weight_copies": (ctypes.c_int, [i32] * 4 + [vp] * 4),
        "lbib_nn_conv3x3_tc_supported": (ctypes.c_int, [i32] * 5),
        "lbib_nn_tile_weights_tc": (ctypes.c_int, [i32, i32, vp, vp, ctypes.POINTER(u64), vp]),
        "lbib_nn_conv3x3_tc": (ctypes.c_int, [i32] * 6 + [vp] * 5 + [i32, i32, vp, vp]),
        "lbib_nn_conv3x3_wgrad_tc_supported": (ctypes.c_int, [i32] * 5),
        "lbib_nn_conv3x3_wgrad_tc": (ctypes.c_int, [i32] * 6 + [vp] * 7),
        "lbib_destroy": (None, [vp]),
        "lbib_last_error": (ctypes.c_char_p, [vp]),
        "lbib_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _status_name(code: int) -> str:
    try:
        return load().lbib_status_string(code).decode()
    except Exception:
        return str(code)


def _check(rc: int, ctx=None):
    if rc != LBIB_OK:
        msg = load().lbib_last_error(ctx).decode(errors="replace")
        raise LbibError(rc, msg)


def _p(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def make_params(p, precision: int = LBIB_FP64) -> lbib_params:
    """lbib_params from any object with the fields of the C struct."""
    o = lbib_params()
    o.nx, o.ny, o.bc_y, o.n_species = int(p.nx), int(p.ny), int(p.bc_y), int(p.n_species)
    o.tau, o.rho0 = float(p.tau), float(p.rho0)
    for s in range(4):
        o.D[s] = float(p.D[s])
        o.decay[s] = float(p.decay[s])
        o.src_rate[s] = float(p.src_rate[s])
        for b in range(4):
            o.react[s][b] = float(p.react[s][b])
    o.forcing = int(getattr(p, "forcing", 0))
    o.precision = int(precision)
    o.fp16_scale = float(getattr(p, "fp16_scale", 0.0) or 0.0)
    o.fp16_scale_species = float(getattr(p, "fp16_scale_species", 0.0) or 0.0)
    o.tension = float(getattr(p, "tension", 0.0) or 0.0)
    bf = getattr(p, "body_force", (0.0, 0.0)) or (0.0, 0.0)
    o.body_force[0], o.body_force[1] = float(bf[0]), float(bf[1])
    o.reaction = int(getattr(p, "reaction", 0) or 0)
    o.noflux_mask = int(getattr(p, "noflux", 0) or 0)
    sk = getattr(p, "schnak", (0.0, 0.0, 0.0)) or (0.0, 0.0, 0.0)
    for q in range(3):
        o.schnak[q] = float(sk[q])
    o.junction_k = float(getattr(p, "junction_k", 0.0) or 0.0)
    o.junction_l0 = float(getattr(p, "junction_l0", 0.0) or 0.0)
    o.junction_lmax = float(getattr(p, "junction_lmax", 0.0) or 0.0)
    o.junction_period = int(getattr(p, "junction_period", 0) or 0)
    o.mass_sources = int(getattr(p, "mass_sources", 0) or 0)
    o.mass_alpha = float(getattr(p, "mass_alpha", 0.0) or 0.0)
    o.pressure_nodes = int(getattr(p, "pressure_nodes", 0) or 0)
    o.pressure_rho = float(getattr(p, "pressure_rho", 0.0) or 0.0)
    o.node_sources = int(getattr(p, "node_sources", 0) or 0)
    o.noflux_scheme = int(getattr(p, "noflux_scheme", 0) or 0)
    if float(getattr(p, "mass_beta", 0.0) or 0.0) != 0.0 or int(getattr(p, "noflux_dynamic", 0) or 0):
        raise ValueError("the concentration-proportional mass source and confinement by moving "
                         "membranes have no CUDA path")
    return o


# ---------------------------------------------------------------- C names
def lbib_workspace_size(params: lbib_params, max_vertices: int, max_cells: int) -> int:
    n = ctypes.c_uint64(0)
    _check(load().lbib_workspace_size(ctypes.byref(params), max_vertices, max_cells, ctypes.byref(n)))
    return int(n.value)


def lbib_create(params: lbib_params, max_vertices: int, max_cells: int, d_workspace: int,
                nbytes: int, stream: int) -> int:
    ctx = ctypes.c_void_p(0)
    _check(load().lbib_create(ctypes.byref(params), max_vertices, max_cells,
                              ctypes.c_void_p(d_workspace), nbytes, ctypes.c_void_p(stream),
                              ctypes.byref(ctx)))
    return ctx.value


def lbib_set_cells(ctx, cell_off, xy, rest_len=None, k_spring=None, pressure=None, src_flag=None):
    off, off_p = _p(cell_off, np.int32)
    xy_, xy_p = _p(xy, np.float64)
    L0, L0_p = _p(rest_len, np.float64)
    k, k_p = _p(k_spring, np.float64)
    pr, pr_p = _p(pressure, np.float64)
    sf, sf_p = _p(src_flag, np.uint8)
    _check(load().lbib_set_cells(ctx, len(off) - 1, off_p, xy_p, L0_p, k_p, pr_p, sf_p), ctx)


def lbib_set_domains(ctx, labels=None):
    """labels: (ny, nx) int32 domain of every node, or None (one domain)."""
    a, a_p = _p(labels, np.int32)
    _check(load().lbib_set_domains(ctx, a_p), ctx)


def lbib_set_mass_sources(ctx, rate=None, target_area=None):
    """rate, target_area: per-cell float64 arrays, or None."""
    r, r_p = _p(rate, np.float64)
    t, t_p = _p(target_area, np.float64)
    _check(load().lbib_set_mass_sources(ctx, r_p, t_p), ctx)


def lbib_set_pressure_nodes(ctx, mask=None):
    """mask: (ny, nx) uint8, nonzero = pressure node, or None (none)."""
    m, m_p = _p(mask, np.uint8)
    _check(load().lbib_set_pressure_nodes(ctx, m_p), ctx)


def lbib_set_node_sources(ctx, S=None):
    """S: (ny, nx) float64 mass source per node, or None (none)."""
    a, a_p = _p(S, np.float64)
    _check(load().lbib_set_node_sources(ctx, a_p), ctx)


def lbib_set_lattice_variant(ctx, nodes_per_thread: int):
    _check(load().lbib_set_lattice_variant(ctx, int(nodes_per_thread)), ctx)


def lbib_get_cells_async(ctx, which: int, xy_ptr, area_ptr):
    """Start the asynchronous readback of the vertex positions (LBIB_X) and /
    or the cell areas (LBIB_AREA) into host buffers given by address (pinned
    for the copy to overlap the next steps); lbib_wait_readback ends it."""
    vp = ctypes.c_void_p
    _check(load().lbib_get_cells_async(ctx, int(which), vp(xy_ptr) if xy_ptr else None,
                                       vp(area_ptr) if area_ptr else None), ctx)


def lbib_wait_readback(ctx):
    _check(load().lbib_wait_readback(ctx), ctx)


def lbib_set_cell_params(ctx, pressure=None, src_flag=None):
    pr, pr_p = _p(pressure, np.float64)
    sf, sf_p = _p(src_flag, np.uint8)
    _check(load().lbib_set_cell_params(ctx, pr_p, sf_p), ctx)


def lbib_set_species(ctx, s: int, phi):
    a, a_p = _p(phi, np.float64)
    _check(load().lbib_set_species(ctx, s, a_p), ctx)


def lbib_step(ctx, n_steps: int):
    _check(load().lbib_step(ctx, int(n_steps)), ctx)


def lbib_advance(ctx, n_steps: int) -> None:
    _check(load().lbib_advance(ctx, int(n_steps)), ctx)


def lbib_get_sums(ctx, n_species: int, n_cells: int):
    """(global (3 + S,), per cell (n_cells, 1 + S), non-finite node count)."""
    glob = np.zeros(3 + n_species)
    cell = np.zeros((max(n_cells, 1), 1 + n_species))
    bad = ctypes.c_uint32(0)
    _check(load().lbib_get_sums(ctx, glob.ctypes.data_as(ctypes.c_void_p),
                                cell.ctypes.data_as(ctypes.c_void_p), ctypes.byref(bad)), ctx)
    return glob, cell[:n_cells], int(bad.value)


def lbib_step_profiled(ctx, n_steps: int):
    """(lattice ms, IB ms) summed over the launches of n_steps steps."""
    ms = np.zeros(2)
    _check(load().lbib_step_profiled(ctx, int(n_steps), ms.ctypes.data_as(ctypes.c_void_p)), ctx)
    return float(ms[0]), float(ms[1])


def lbib_get_fields(ctx, which: int, nx: int, ny: int, n_species: int, n_vertices: int,
                    n_cells: int) -> dict:
    out = {}

    def buf(key, shape, dtype=np.float64, flag=0):
        if which & flag:
            out[key] = np.empty(shape, dtype)
            return out[key].ctypes.data_as(ctypes.c_void_p)
        return None

    rho = buf("rho", (ny, nx), flag=LBIB_RHO)
    ux = buf("ux", (ny, nx), flag=LBIB_U)
    uy = buf("uy", (ny, nx), flag=LBIB_U)
    phi = buf("phi", (max(n_species, 1), ny, nx), flag=LBIB_PHI)
    xy = buf("xy", (max(n_vertices, 1), 2), flag=LBIB_X)
    area = buf("area", (max(n_cells, 1),), flag=LBIB_AREA)
    idp = buf("id", (ny, nx), np.int32, flag=LBIB_ID)
    force = buf("force", (ny, nx, 2), flag=LBIB_FORCE)
    vf = buf("vforce", (max(n_vertices, 1), 2), flag=LBIB_VFORCE)
    _check(load().lbib_get_fields(ctx, which, rho, ux, uy, phi, xy, area, idp, force, vf), ctx)
    if "phi" in out:
        out["phi"] = out["phi"][:n_species]
    for k, n in (("xy", n_vertices), ("vforce", n_vertices), ("area", n_cells)):
        if k in out:
            out[k] = out[k][:n]
    return out


def lbib_get_sizes(ctx):
    v, c = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().lbib_get_sizes(ctx, ctypes.byref(v), ctypes.byref(c)), ctx)
    return v.value, c.value


def lbib_state_size(ctx) -> int:
    n = ctypes.c_uint64(0)
    _check(load().lbib_state_size(ctx, ctypes.byref(n)), ctx)
    return int(n.value)


def lbib_get_state(ctx) -> np.ndarray:
    n = lbib_state_size(ctx)
    buf = np.empty(n, np.uint8)
    _check(load().lbib_get_state(ctx, buf.ctypes.data_as(ctypes.c_void_p), n), ctx)
    return buf


def lbib_set_state(ctx, state: np.ndarray):
    b = np.ascontiguousarray(state, np.uint8)
    _check(load().lbib_set_state(ctx, b.ctypes.data_as(ctypes.c_void_p), b.size), ctx)


def lbib_step_noalloc(params: lbib_params, n_cells: int, d_cell_off: int, d_xy: int,
                      d_rest_len: int, d_k_spring: int, d_pressure: int, d_src_flag: int,
                      d_f: int, d_g: int, n_steps: int, stream: int):
    """Allocation-free coupled steps on caller-owned device buffers (raw
    device addresses); see include/lbib.h for the buffer layout."""
    vp = ctypes.c_void_p
    _check(load().lbib_step_noalloc(ctypes.byref(params), n_cells, vp(d_cell_off), vp(d_xy),
                                    vp(d_rest_len), vp(d_k_spring), vp(d_pressure),
                                    vp(d_src_flag), vp(d_f), vp(d_g), int(n_steps),
                                    vp(stream)))


def lbib_label_cells(nx: int, ny: int, bc_y: int, n_cells: int, d_cell_off: int, d_xy: int,
                     d_src_flag: int, d_id: int, d_src: int, stream: int):
    vp = ctypes.c_void_p
    _check(load().lbib_label_cells(nx, ny, bc_y, n_cells, vp(d_cell_off), vp(d_xy),
                                   vp(d_src_flag), vp(d_id), vp(d_src or None), vp(stream)))


def lbib_steady_workspace_size(nx: int, ny: int, batch: int) -> int:
    n = ctypes.c_uint64(0)
    _check(load().lbib_steady_workspace_size(nx, ny, batch, ctypes.byref(n)))
    return int(n.value)


def lbib_steady_solve(nx, ny, batch, d_src, D, decay, src_rate, d_phi0, tol, max_steps,
                      check_every, d_phi_out, d_workspace, ws_bytes, stream):
    """Returns (steps, resid, fallback) host arrays; d_* are raw device
    addresses.  fallback[b] = 1 where a warm start was abandoned."""
    vp = ctypes.c_void_p
    D_, Dp = _p(D, np.float64)
    k_, kp = _p(decay, np.float64)
    s_, sp = _p(src_rate, np.float64)
    steps = np.zeros(batch, np.int64)
    resid = np.zeros(batch, np.float64)
    fallback = np.zeros(batch, np.int32)
    _check(load().lbib_steady_solve(nx, ny, batch, vp(d_src), Dp, kp, sp, vp(d_phi0 or None),
                                    float(tol), int(max_steps), int(check_every), vp(d_phi_out),
                                    steps.ctypes.data_as(vp), resid.ctypes.data_as(vp),
                                    fallback.ctypes.data_as(vp), vp(d_workspace), int(ws_bytes),
                                    vp(stream)))
    return steps, resid, fallback


def steady_solve(src, D, decay, src_rate, phi0=None, tol=1e-6, max_steps=200000,
                 check_every=16, stream=None, with_fallback=False):
    """Convenience wrapper on torch CUDA tensors: src (B, ny, nx) uint8,
    phi0 (B, ny, nx) float32 or None.  Returns (phi, steps, resid), plus the
    per-tissue fallback flags with with_fallback."""
    import torch
    B, ny, nx = src.shape
    ws_n = lbib_steady_workspace_size(nx, ny, B)
    ws = torch.empty(ws_n, dtype=torch.uint8, device=src.device)
    out = torch.empty((B, ny, nx), dtype=torch.float32, device=src.device)
    st = (stream or torch.cuda.current_stream(src.device)).cuda_stream
    src = src.contiguous()
    p0 = None if phi0 is None else phi0.contiguous().float()
    steps, resid, fb = lbib_steady_solve(nx, ny, B, src.data_ptr(), D, decay, src_rate,
                                         None if p0 is None else p0.data_ptr(), tol, max_steps,
                                         check_every, out.data_ptr(), ws.data_ptr(), ws_n, st)
    if with_fallback:
        return out, steps, resid, fb
    return out, steps, resid


def label_cells(nx, ny, bc_y, tissue, device="cuda"):
    """Labels of a host tissue, computed on the device.  Returns (id, src)
    torch tensors (ny, nx)."""
    import torch
    off = torch.as_tensor(np.ascontiguousarray(tissue.cell_off, np.int32), device=device)
    xy = torch.as_tensor(np.ascontiguousarray(tissue.xy, np.float64), device=device)
    sf = torch.as_tensor(np.ascontiguousarray(tissue.src_flag, np.uint8), device=device)
    idt = torch.empty((ny, nx), dtype=torch.int32, device=device)
    srt = torch.empty((ny, nx), dtype=torch.uint8, device=device)
    lbib_label_cells(nx, ny, bc_y, tissue.n_cells, off.data_ptr(), xy.data_ptr(), sf.data_ptr(),
                     idt.data_ptr(), srt.data_ptr(), torch.cuda.current_stream(device).cuda_stream)
    return idt, srt


def lbib_destroy(ctx):
    if ctx:
        load().lbib_destroy(ctx)


def lbib_last_error(ctx=None) -> str:
    return load().lbib_last_error(ctx).decode(errors="replace")


def lbib_status_string(code: int) -> str:
    return load().lbib_status_string(code).decode()


# ---------------------------------------------------------------- convenience
class Simulation:
    """One tissue on one GPU.  The workspace is a torch uint8 CUDA tensor
    owned by this object; the stream defaults to torch's current stream."""

    def __init__(self, params, precision: int = LBIB_FP64, max_vertices: int = 0,
                 max_cells: int = 0, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("lbib needs a CUDA device; there is no CPU path")
        load()
        self.device = torch.device(device or "cuda")
        self.cparams = make_params(params, precision)
        self.nx, self.ny = int(params.nx), int(params.ny)
        self.n_species = int(params.n_species)
        self.nbytes = lbib_workspace_size(self.cparams, max_vertices, max_cells)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.ctx = lbib_create(self.cparams, max_vertices, max_cells, self.workspace.data_ptr(),
                               self.nbytes, self.stream.cuda_stream)
        self.n_vertices = 0
        self.n_cells = 0

    def set_cells(self, tissue=None, **kw):
        if tissue is not None:
            kw = dict(cell_off=tissue.cell_off, xy=tissue.xy, rest_len=tissue.rest_len,
                      k_spring=tissue.k_spring, pressure=tissue.pressure,
                      src_flag=tissue.src_flag)
        lbib_set_cells(self.ctx, **kw)
        self.n_vertices, self.n_cells = lbib_get_sizes(self.ctx)

    def set_cell_params(self, pressure=None, src_flag=None):
        lbib_set_cell_params(self.ctx, pressure, src_flag)

    def set_domains(self, labels=None):
        lbib_set_domains(self.ctx, labels)

    def set_mass_sources(self, rate=None, target_area=None):
        lbib_set_mass_sources(self.ctx, rate, target_area)

    def set_pressure_nodes(self, mask=None):
        lbib_set_pressure_nodes(self.ctx, mask)

    def set_node_sources(self, S=None):
        lbib_set_node_sources(self.ctx, S)

    def set_lattice_variant(self, nodes_per_thread: int):
        lbib_set_lattice_variant(self.ctx, nodes_per_thread)

    def set_species(self, s: int, phi):
        lbib_set_species(self.ctx, s, phi)

    def step(self, n: int = 1):
        lbib_step(self.ctx, n)

    def sums(self):
        """FP64 conservation sums of the last step (lbib_get_sums)."""
        return lbib_get_sums(self.ctx, self.n_species, self.n_cells)

    def advance(self, n: int = 1):
        """n steps without the output work of the last one (lbib_advance)."""
        lbib_advance(self.ctx, n)

    def step_profiled(self, n: int):
        return lbib_step_profiled(self.ctx, n)

    def fields(self, which: int = LBIB_RHO | LBIB_U | LBIB_PHI | LBIB_X) -> dict:
        if self.n_species == 0:
            which &= ~LBIB_PHI
        if self.n_cells == 0:
            which &= ~(LBIB_X | LBIB_AREA | LBIB_ID | LBIB_FORCE | LBIB_VFORCE)
        return lbib_get_fields(self.ctx, which, self.nx, self.ny, self.n_species,
                               self.n_vertices, self.n_cells)

    def get_state(self) -> np.ndarray:
        return lbib_get_state(self.ctx)

    def set_state(self, st):
        lbib_set_state(self.ctx, st)
        self.n_vertices, self.n_cells = lbib_get_sizes(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            lbib_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- ensembles
def _ens_check(rc, ens):
    if rc != LBIB_OK:
        raise LbibError(rc, load().lbib_ensemble_last_error(ens).decode(errors="replace"))


class Ensemble:
    """Many independent FP32 tissues advanced by one persistent launch per
    step call, or by two launches per step (the split schedules).  ``params``
    is a list of parameter objects; ``tissues`` the matching list of tissues
    (lbib_inputs.Tissue-like; None for a tissue without cells)."""

    def __init__(self, params, tissues, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("lbib needs a CUDA device; there is no CPU path")
        L = load()
        self.device = torch.device(device or "cuda")
        n = len(params)
        self.n = n
        arr = (lbib_params * n)(*[make_params(p, LBIB_FP32) for p in params])
        self._params = arr
        self.dims = [(int(p.nx), int(p.ny), int(p.n_species)) for p in params]
        mv = np.array([t.n_vertices if t is not None else 0 for t in tissues], np.int32)
        mc = np.array([t.n_cells if t is not None else 0 for t in tissues], np.int32)
        nb = ctypes.c_uint64(0)
        vp = ctypes.c_void_p
        _ens_check(L.lbib_ensemble_workspace_size(n, arr, mv.ctypes.data_as(vp),
                                                  mc.ctypes.data_as(vp), ctypes.byref(nb)), None)
        self.nbytes = int(nb.value)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p(0)
        _ens_check(L.lbib_ensemble_create(n, arr, mv.ctypes.data_as(vp), mc.ctypes.data_as(vp),
                                          vp(self.workspace.data_ptr()), self.nbytes,
                                          vp(self.stream.cuda_stream), ctypes.byref(h)), None)
        self.ens = h.value
        self.ctx = [L.lbib_ensemble_tissue(self.ens, t) for t in range(n)]
        self.sizes = [(0, 0)] * n
        for t, T in enumerate(tissues):
            if T is not None and T.n_cells:
                lbib_set_cells(self.ctx[t], T.cell_off, T.xy, T.rest_len, T.k_spring,
                               T.pressure, T.src_flag)
                self.sizes[t] = lbib_get_sizes(self.ctx[t])

    def step(self, n: int):
        _ens_check(load().lbib_ensemble_step(self.ens, int(n)), self.ens)

    def status(self):
        _ens_check(load().lbib_ensemble_status(self.ens), self.ens)

    def config(self, nodes_per_item: int = 0, blocks_per_sm: int = -1):
        g, gr = ctypes.c_int32(0), ctypes.c_int32(0)
        _ens_check(load().lbib_ensemble_config(self.ens, nodes_per_item, blocks_per_sm,
                                               ctypes.byref(g), ctypes.byref(gr)), self.ens)
        return {"graph": bool(g.value), "grid": int(gr.value)}

    def schedule(self, schedule: int = -1) -> int:
        """Set the schedule (LBIB_ENS_PERSISTENT / LBIB_ENS_SPLIT /
        LBIB_ENS_SPLIT_WIDE; < 0 keeps it); returns the one in use."""
        out = ctypes.c_int32(0)
        _ens_check(load().lbib_ensemble_schedule(self.ens, int(schedule), ctypes.byref(out)),
                   self.ens)
        return int(out.value)

    def tune(self, trial_steps: int = 20):
        cfg = np.zeros(2, np.int32)
        ms = ctypes.c_double(0.0)
        _ens_check(load().lbib_ensemble_tune(self.ens, int(trial_steps),
                                             cfg.ctypes.data_as(ctypes.c_void_p),
                                             ctypes.byref(ms)), self.ens)
        return {"nodes_per_item": int(cfg[0]), "blocks_per_sm": int(cfg[1]),
                "schedule": self.schedule(), "ms_per_step": float(ms.value)}

    def tune_cached(self, key: str, trial_steps: int = 20, path: Optional[str] = None):
        """Autotune once per ``key`` and keep the choice in a JSON cache
        (``$LBIB_TUNE_CACHE`` or ~/.cache/lbib_tune.json)."""
        import json
        path = path or os.environ.get("LBIB_TUNE_CACHE",
                                      os.path.join(os.path.expanduser("~"), ".cache",
                                                   "lbib_tune.json"))
        cache = {}
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            c = cache[key]
            self.config(c["nodes_per_item"], c["blocks_per_sm"])
            self.schedule(c.get("schedule", LBIB_ENS_PERSISTENT))
            return dict(c, cached=True)
        c = self.tune(trial_steps)
        cache[key] = c
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
        return dict(c, cached=False)

    def selftest_timeout(self):
        sec = ctypes.c_double(0.0)
        rc = load().lbib_ensemble_selftest_timeout(self.ens, ctypes.byref(sec))
        return rc, float(sec.value)

    def fields(self, t: int, which: int = LBIB_RHO | LBIB_U | LBIB_PHI | LBIB_X) -> dict:
        nx, ny, S = self.dims[t]
        nv, nc = self.sizes[t]
        if S == 0:
            which &= ~LBIB_PHI
        if nc == 0:
            which &= ~(LBIB_X | LBIB_AREA | LBIB_ID | LBIB_FORCE | LBIB_VFORCE)
        return lbib_get_fields(self.ctx[t], which, nx, ny, S, nv, nc)

    def close(self):
        if getattr(self, "ens", None):
            load().lbib_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- neural operator
def _nop_check(rc, h):
    if rc != LBIB_OK:
        raise LbibError(rc, load().lbib_nop_last_error(h).decode(errors="replace"))


class NeuralOperator:
    """The U-Net warm start (include/lbib.h, neural operator section) on a
    torch-owned workspace."""

    def __init__(self, batch: int, H: int = 256, W: int = 256, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("lbib needs a CUDA device; there is no CPU path")
        L = load()
        self.device = torch.device(device or "cuda")
        self.B, self.H, self.W = batch, H, W
        nb = ctypes.c_uint64(0)
        _nop_check(L.lbib_nop_workspace_size(batch, H, W, ctypes.byref(nb)), None)
        self.nbytes = int(nb.value)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p(0)
        _nop_check(L.lbib_nop_create(batch, H, W, ctypes.c_void_p(self.workspace.data_ptr()),
                                     self.nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.byref(h)), None)
        self.h = h.value
        n = ctypes.c_int64(0)
        _nop_check(L.lbib_nop_num_params(self.h, ctypes.byref(n)), self.h)
        self.n_params = int(n.value)

    def layers(self):
        L = load()
        n = ctypes.c_int32(0)
        _nop_check(L.lbib_nop_layers(self.h, ctypes.byref(n), None), self.h)
        cc = np.zeros(2 * n.value, np.int32)
        _nop_check(L.lbib_nop_layers(self.h, ctypes.byref(n), cc.ctypes.data_as(ctypes.c_void_p)),
                   self.h)
        return [(int(cc[2 * i]), int(cc[2 * i + 1])) for i in range(n.value)]

    def set_params(self, p):
        a = np.ascontiguousarray(p, np.float32)
        _nop_check(load().lbib_nop_set_params(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size),
                   self.h)

    def get_params(self):
        a = np.empty(self.n_params, np.float32)
        _nop_check(load().lbib_nop_get_params(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size),
                   self.h)
        return a

    def get_grads(self):
        a = np.empty(self.n_params, np.float32)
        _nop_check(load().lbib_nop_get_grads(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size),
                   self.h)
        return a

    def forward(self, mask, src, D, decay, src_rate, out=None):
        """mask, src: (n, H, W) uint8 CUDA tensors; returns phi (n, H, W) float32."""
        import torch
        n = mask.shape[0]
        if out is None:
            out = torch.empty((n, self.H, self.W), dtype=torch.float32, device=mask.device)
        _, Dp = _p(D, np.float64)
        _, kp = _p(decay, np.float64)
        _, sp = _p(src_rate, np.float64)
        keep = (_, Dp, kp, sp)
        _nop_check(load().lbib_nop_forward(self.h, n, ctypes.c_void_p(mask.data_ptr()),
                                           ctypes.c_void_p(src.data_ptr()), Dp, kp, sp,
                                           ctypes.c_void_p(out.data_ptr())), self.h)
        del keep
        return out

    def train_step(self, mask, src, D, decay, src_rate, phi, lr=1e-3, update=True):
        n = mask.shape[0]
        Da = np.ascontiguousarray(D, np.float64)
        ka = np.ascontiguousarray(decay, np.float64)
        sa = np.ascontiguousarray(src_rate, np.float64)
        loss = ctypes.c_double(0.0)
        vp = ctypes.c_void_p
        _nop_check(load().lbib_nop_train_step(self.h, n, vp(mask.data_ptr()), vp(src.data_ptr()),
                                              Da.ctypes.data_as(vp), ka.ctypes.data_as(vp),
                                              sa.ctypes.data_as(vp), vp(phi.data_ptr()),
                                              float(lr), 1 if update else 0,
                                              ctypes.byref(loss)), self.h)
        return float(loss.value)

    def close(self):
        if getattr(self, "h", None):
            load().lbib_nop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
