"""FP64 CPU oracle of the LBIBCell coupled step -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It compiles ``lbib_oracle.c`` (plain C, FP64, no FMA
contraction) with gcc into ``oracle/_build/liblbib_oracle.so`` and exposes
numpy-level wrappers.  It shares no code with the CUDA library.

Parity status per function (what pins it; see tests/test_oracle_pins.py):
  delta1d            partition of unity, second-moment sum 3/8, symmetry
  polygon_forces     zero net force, regular n-gon closed form, rest state
  cell_areas         regular n-gon closed form, translation invariance
  rasterize          brute-force point-in-circle counts, shifted copies
  spread / interp    total force, adjointness, constant-field interpolation
  lattice_step       mass and momentum budgets, equilibrium fixed point,
                     Poiseuille curvature, Taylor-Green decay
  species_step       mass budget with decay and source, Green's function
                     variance growth 2Dt
  run (coupled)      invariants above; the coupled trajectory itself is
                     parity unpinned beyond them (no printed trajectory)
  sums               global mass conserved on a periodic lattice, global
                     momentum (n - 1/2) N F under a uniform body force F,
                     per-cell sums adding up to the sum over labelled nodes
  steady             closed-form uniform steady state s/k
  Schnakenberg       homogeneous fixed point (a+b, b/(a+b)^2), linearised
    reaction         map I + J of a uniform perturbation (Jacobian by hand)
  junctions          two facing polygons: partners and force k (g - l0) across
                     a gap g by construction, nothing beyond l_max, the
                     periodic image, equal and opposite forces of mutual pairs
  no-flux closure    the paper's equilibrium closure (Sec. 6.1): closed form
    (scheme 0)       for a linear density and a given momentum, the thin-
                     domain fallbacks, rotation and mirror invariance, uniform
                     domains as a fixed point with an empty domain staying
                     empty, first-order convergence to the closed-form
                     Neumann profile with no steady leak, first-order decay
                     of the transient leak with straight membranes
  bounce-back        per-domain mass conservation of a confined species (a
    (scheme 1)       free one moves mass), relaxation to the domain mean;
                     either scheme: one label everywhere = no confinement
  conv3x3 (+dgrad,   scipy correlate2d, identity tap, adjointness,
    wgrad)           finite differences
  nn (U-Net)         finite-difference gradient of the whole network,
                     pooling/upsampling adjoints, Adam first-step closed form
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbib_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbib_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc_y", ctypes.c_int32),
                ("n_species", ctypes.c_int32), ("tau", ctypes.c_double),
                ("rho0", ctypes.c_double), ("D", ctypes.c_double * 4),
                ("decay", ctypes.c_double * 4), ("react", (ctypes.c_double * 4) * 4),
                ("src_rate", ctypes.c_double * 4), ("forcing", ctypes.c_int32),
                ("react_model", ctypes.c_int32), ("noflux", ctypes.c_int32),
                ("noflux_scheme", ctypes.c_int32), ("schnak", ctypes.c_double * 3),
                ("junction_k", ctypes.c_double), ("junction_l0", ctypes.c_double),
                ("junction_lmax", ctypes.c_double), ("junction_period", ctypes.c_int32),
                ("pad2", ctypes.c_int32), ("mass_alpha", ctypes.c_double),
                ("pressure_rho", ctypes.c_double), ("mass_beta", ctypes.c_double),
                ("mass_species", ctypes.c_int32), ("noflux_dynamic", ctypes.c_int32)]


def _P(p) -> OrcParams:
    o = OrcParams()
    o.nx, o.ny, o.bc_y, o.n_species = int(p.nx), int(p.ny), int(p.bc_y), int(p.n_species)
    o.tau, o.rho0 = float(p.tau), float(p.rho0)
    for s in range(4):
        o.D[s] = float(p.D[s])
        o.decay[s] = float(p.decay[s])
        o.src_rate[s] = float(p.src_rate[s])
        for b in range(4):
            o.react[s][b] = float(p.react[s][b])
    o.forcing = int(p.forcing)
    o.react_model = int(getattr(p, "reaction", 0))
    o.noflux = int(getattr(p, "noflux", 0))
    o.noflux_scheme = int(getattr(p, "noflux_scheme", 0) or 0)
    sk = getattr(p, "schnak", (0.0, 0.0, 0.0))
    for q in range(3):
        o.schnak[q] = float(sk[q])
    o.junction_k = float(getattr(p, "junction_k", 0.0))
    o.junction_l0 = float(getattr(p, "junction_l0", 0.0))
    o.junction_lmax = float(getattr(p, "junction_lmax", 0.0))
    o.junction_period = int(getattr(p, "junction_period", 0))
    o.mass_alpha = float(getattr(p, "mass_alpha", 0.0))
    o.pressure_rho = float(getattr(p, "pressure_rho", 0.0))
    o.mass_beta = float(getattr(p, "mass_beta", 0.0))
    o.mass_species = int(getattr(p, "mass_species", 0))
    o.noflux_dynamic = int(getattr(p, "noflux_dynamic", 0))
    return o


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d = ctypes.c_double
            vp = ctypes.c_void_p
            i = ctypes.c_int
            L.orc_delta1d.restype = d
            L.orc_delta1d.argtypes = [d]
            L.orc_polygon_forces.argtypes = [i, vp, vp, vp, vp, vp, vp]
            L.orc_tension_forces.argtypes = [i, vp, vp, d, vp]
            L.orc_cell_areas.argtypes = [i, vp, vp, vp]
            L.orc_junction_partners.argtypes = [i, i, i, i, vp, vp, d, vp]
            L.orc_junction_forces.argtypes = [i, i, i, i, vp, vp, d, d, d, vp]
            L.orc_rasterize.argtypes = [i, i, i, i, vp, vp, vp, vp, vp]
            L.orc_spread.argtypes = [i, i, i, i, vp, vp, vp, vp]
            L.orc_interp.argtypes = [i, i, i, i, vp, vp, vp, vp]
            L.orc_lattice_step.argtypes = [ctypes.POINTER(OrcParams)] + [vp] * 17
            L.orc_species_step.argtypes = [ctypes.POINTER(OrcParams)] + [vp] * 9
            L.orc_species_moments.argtypes = [ctypes.POINTER(OrcParams), vp, vp]
            L.orc_run.restype = i
            L.orc_run.argtypes = ([ctypes.POINTER(OrcParams), i, vp, vp, vp, vp, vp, d, vp, i]
                                  + [vp] * 17)
            L.orc_steady.restype = ctypes.c_long
            L.orc_steady.argtypes = [ctypes.POINTER(OrcParams), vp, vp, d, ctypes.c_long, i,
                                     vp, ctypes.POINTER(d)]
            L.orc_conv3x3.argtypes = [i, i, i, i, i, vp, vp, vp, vp]
            L.orc_conv3x3_dgrad.argtypes = [i, i, i, i, i, vp, vp, vp]
            L.orc_conv3x3_wgrad.argtypes = [i, i, i, i, i, vp, vp, vp, vp]
            L.orc_set_threads.argtypes = [i]
            L.orc_max_threads.restype = i
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def delta1d(r: float) -> float:
    return float(lib().orc_delta1d(float(r)))


def polygon_forces(cell_off, xy, L0, k, p, tension: float = 0.0) -> np.ndarray:
    off = np.ascontiguousarray(cell_off, np.int32)
    xy = _f64(xy)
    F = np.zeros_like(xy)
    lib().orc_polygon_forces(len(off) - 1, _ptr(off), _ptr(xy), _ptr(_f64(L0)), _ptr(_f64(k)),
                             _ptr(_f64(p)), _ptr(F))
    if tension:
        lib().orc_tension_forces(len(off) - 1, _ptr(off), _ptr(xy), float(tension), _ptr(F))
    return F


def junction_partners(nx, ny, bc_y, cell_off, xy, lmax) -> np.ndarray:
    off = np.ascontiguousarray(cell_off, np.int32)
    xy = _f64(xy)
    partner = np.zeros(xy.shape[0], np.int32)
    lib().orc_junction_partners(nx, ny, bc_y, len(off) - 1, _ptr(off), _ptr(xy), float(lmax),
                                _ptr(partner))
    return partner


def junction_forces(nx, ny, bc_y, xy, partner, k, l0, lmax) -> np.ndarray:
    xy = _f64(xy)
    F = np.zeros_like(xy)
    lib().orc_junction_forces(nx, ny, bc_y, xy.shape[0], _ptr(xy),
                              _ptr(np.ascontiguousarray(partner, np.int32)), float(k), float(l0),
                              float(lmax), _ptr(F))
    return F


def cell_areas(cell_off, xy) -> np.ndarray:
    off = np.ascontiguousarray(cell_off, np.int32)
    a = np.zeros(len(off) - 1)
    lib().orc_cell_areas(len(off) - 1, _ptr(off), _ptr(_f64(xy)), _ptr(a))
    return a


def rasterize(nx, ny, bc_y, cell_off, xy, src_flag):
    off = np.ascontiguousarray(cell_off, np.int32)
    idp = np.zeros((ny, nx), np.int32)
    src = np.zeros((ny, nx), np.uint8)
    lib().orc_rasterize(nx, ny, bc_y, len(off) - 1, _ptr(off), _ptr(_f64(xy)),
                        _ptr(np.ascontiguousarray(src_flag, np.uint8)), _ptr(idp), _ptr(src))
    return idp, src


def spread(nx, ny, bc_y, xy, F):
    xy = _f64(xy)
    fx = np.zeros((ny, nx))
    fy = np.zeros((ny, nx))
    lib().orc_spread(nx, ny, bc_y, xy.shape[0], _ptr(xy), _ptr(_f64(F)), _ptr(fx), _ptr(fy))
    return fx, fy


def interp(nx, ny, bc_y, xy, ux, uy):
    xy = _f64(xy)
    U = np.zeros_like(xy)
    lib().orc_interp(nx, ny, bc_y, xy.shape[0], _ptr(xy), _ptr(_f64(ux)), _ptr(_f64(uy)),
                     _ptr(U))
    return U


W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W5 = np.array([1 / 3] + [1 / 6] * 4)


def equilibrium_state(p):
    """Populations at rest: f = w rho0, g = 0 (the initial state)."""
    N = p.nx * p.ny
    f = np.repeat(W9 * p.rho0, N).reshape(9, p.ny, p.nx).copy()
    g = np.zeros((p.n_species * 5, p.ny, p.nx))
    return f, g


def _dom(dom):
    return None if dom is None else np.ascontiguousarray(dom, np.int32)


def _opt(a, dt):
    return None if a is None else np.ascontiguousarray(a, dt)


def species_moments(p, g):
    """Density and momentum (phi, jx, jy) of every species from populations
    g at the same node: (3S, ny, nx).  The moments a run starts from."""
    P = _P(p)
    mom = np.empty((3 * p.n_species, p.ny, p.nx))
    lib().orc_species_moments(ctypes.byref(P), _ptr(_f64(g)), _ptr(mom))
    return mom


def _mom_in(p, g, mom, dom):
    """The previous step's species moments for the no-flux closure (only
    needed with confined species): given, or those of g."""
    if not (p.n_species and int(getattr(p, "noflux", 0)) and dom is not None):
        return None
    return species_moments(p, g) if mom is None else _f64(mom)


def lattice_step(p, f, g, fx=None, fy=None, src=None, dom=None, msrc=None, pmask=None,
                 lab=None, mom=None, mom_out=None):
    """One stream+collide update.  Returns (f_out, g_out, rho, ux, uy, phi).
    dom: static domain labels (ny, nx) for the species confined by p.noflux;
    msrc: mass source per node (ny, nx); pmask: internal pressure nodes
    (ny, nx), prescribed density p.pressure_rho; lab: cell labels (ny, nx),
    > 0 inside a cell, for the source p.mass_beta phi_s.  mom: the species
    moments of the previous step (3S, ny, nx) for the no-flux closure
    (default: those of g); mom_out (3S, ny, nx), if given, receives this
    step's."""
    P = _P(p)
    f = _f64(f)
    g = _f64(g) if p.n_species else np.zeros(1)
    fo = np.empty_like(f)
    go = np.empty_like(g)
    rho = np.empty((p.ny, p.nx))
    ux = np.empty_like(rho)
    uy = np.empty_like(rho)
    phi = np.empty((max(p.n_species, 1), p.ny, p.nx))
    mi = _mom_in(p, g, mom, dom)
    lib().orc_lattice_step(ctypes.byref(P), _ptr(f), _ptr(fo), _ptr(g), _ptr(go),
                           _ptr(None if fx is None else _f64(fx)),
                           _ptr(None if fy is None else _f64(fy)),
                           _ptr(None if src is None else np.ascontiguousarray(src, np.uint8)),
                           _ptr(rho), _ptr(ux), _ptr(uy), _ptr(phi), _ptr(_dom(dom)),
                           _ptr(_opt(msrc, np.float64)), _ptr(_opt(pmask, np.uint8)),
                           _ptr(_opt(lab, np.int32)), _ptr(mi), _ptr(mom_out))
    return fo, go, rho, ux, uy, phi[: p.n_species]


def species_step(p, g, src=None, ux=None, uy=None, dom=None, mom=None, mom_out=None):
    """One D2Q5 update of every species with a frozen velocity (u = 0 when
    ux, uy are None).  Returns (g_out, phi).  dom, mom, mom_out as for
    lattice_step."""
    P = _P(p)
    g = _f64(g)
    go = np.empty_like(g)
    phi = np.empty((p.n_species, p.ny, p.nx))
    mi = _mom_in(p, g, mom, dom)
    lib().orc_species_step(ctypes.byref(P), _ptr(g), _ptr(go),
                           _ptr(None if ux is None else _f64(ux)),
                           _ptr(None if uy is None else _f64(uy)),
                           _ptr(None if src is None else np.ascontiguousarray(src, np.uint8)),
                           _ptr(phi), _ptr(_dom(dom)), _ptr(mi), _ptr(mom_out))
    return go, phi


class RunResult:
    pass


def run(p, tissue, n_steps, f=None, g=None, xy=None, tension: float = 0.0, dom=None,
        mass_rate=None, target_area=None, pmask=None, node_source=None, mom=None):
    """n coupled steps from (f, g, xy) (default: rest state and tissue.xy).
    Returns a RunResult with the final state and the last step's fields.
    dom: static domain labels (ny, nx) for the species confined by p.noflux;
    mass_rate (per cell): mass source of the cell's nodes, plus
    p.mass_alpha (target_area - area) with target_area (per cell); pmask:
    internal pressure nodes (ny, nx) held at density p.pressure_rho;
    node_source: static mass source per node (ny, nx), added to the cells';
    mom: the species moments of the previous step (3S, ny, nx) for the no-flux
    closure of confined species (default: those of the initial g); the
    result's r.mom carries them on to a following call."""
    P = _P(p)
    N = p.nx * p.ny
    if f is None or g is None:
        f0, g0 = equilibrium_state(p)
        f = f0 if f is None else f
        g = g0 if g is None else g
    f = _f64(f).copy()
    g = _f64(g).copy() if p.n_species else np.zeros(1)
    xy = _f64(tissue.xy if xy is None else xy).copy()
    off = np.ascontiguousarray(tissue.cell_off, np.int32)
    r = RunResult()
    r.rho = np.zeros((p.ny, p.nx))
    r.ux = np.zeros_like(r.rho)
    r.uy = np.zeros_like(r.rho)
    r.phi = np.zeros((max(p.n_species, 1), p.ny, p.nx))
    r.id = np.zeros((p.ny, p.nx), np.int32)
    r.src = np.zeros((p.ny, p.nx), np.uint8)
    r.fx = np.zeros_like(r.rho)
    r.fy = np.zeros_like(r.rho)
    V = xy.shape[0]
    r.Fv = np.zeros((max(V, 1), 2))
    r.mom = None
    if p.n_species and int(getattr(p, "noflux", 0)):
        r.mom = species_moments(p, g) if mom is None else _f64(mom).copy()
    rc = lib().orc_run(ctypes.byref(P), len(off) - 1, _ptr(off), _ptr(xy), _ptr(_f64(tissue.rest_len)),
                       _ptr(_f64(tissue.k_spring)), _ptr(_f64(tissue.pressure)), float(tension),
                       _ptr(np.ascontiguousarray(tissue.src_flag, np.uint8)), int(n_steps),
                       _ptr(f), _ptr(g), _ptr(r.rho), _ptr(r.ux), _ptr(r.uy), _ptr(r.phi),
                       _ptr(r.id), _ptr(r.src), _ptr(r.fx), _ptr(r.fy), _ptr(r.Fv),
                       _ptr(_dom(dom)), _ptr(_opt(mass_rate, np.float64)),
                       _ptr(_opt(target_area, np.float64)), _ptr(_opt(pmask, np.uint8)),
                       _ptr(_opt(node_source, np.float64)), _ptr(r.mom))
    if rc != 0:
        raise MemoryError("oracle run failed to allocate")
    r.f = f
    r.g = g
    r.xy = xy
    r.phi = r.phi[: p.n_species]
    r.area = cell_areas(off, xy)
    assert N == p.nx * p.ny
    return r


def sums(p, r, n_cells):
    """Conservation sums of a run's last-step fields (Sec. 3.3 computeAreas
    gives the per-cell area; these are its mass and concentration
    companions), in FP64: global sum rho, sum rho ux, sum rho uy and sum phi_s
    over all nodes; per cell c (the nodes whose lowest containing cell is c,
    id == c + 1) sum rho and sum phi_s.  Returns (glob (3 + S,),
    cell (n_cells, 1 + S))."""
    S = p.n_species
    glob = np.array([r.rho.sum(), (r.rho * r.ux).sum(), (r.rho * r.uy).sum()] +
                    [r.phi[s].sum() for s in range(S)])
    cell = np.zeros((n_cells, 1 + S))
    for c in range(n_cells):
        m = r.id == c + 1
        cell[c, 0] = r.rho[m].sum()
        for s in range(S):
            cell[c, 1 + s] = r.phi[s][m].sum()
    return glob, cell


def steady(p, src, g=None, tol=1e-6, max_steps=200000, check_every=16):
    """Steady D2Q5 solve with u = 0.  Returns (phi, steps, resid, g)."""
    P = _P(p)
    if g is None:
        g = np.zeros((p.n_species * 5, p.ny, p.nx))
    g = _f64(g).copy()
    phi = np.zeros((p.n_species, p.ny, p.nx))
    r = ctypes.c_double(0.0)
    n = lib().orc_steady(ctypes.byref(P), _ptr(np.ascontiguousarray(src, np.uint8)), _ptr(g),
                         float(tol), int(max_steps), int(check_every), _ptr(phi), ctypes.byref(r))
    return phi, int(n), float(r.value), g


# ---------------------------------------------------------------- conv layers
def conv3x3(x, w, b=None):
    """x (N,H,W,Ci), w (3,3,Ci,Co), b (Co,) -> (N,H,W,Co); zero padding."""
    x = _f64(x)
    w = _f64(w)
    N, H, W, Ci = x.shape
    Co = w.shape[3]
    out = np.empty((N, H, W, Co))
    lib().orc_conv3x3(N, H, W, Ci, Co, _ptr(x), _ptr(w), _ptr(None if b is None else _f64(b)),
                      _ptr(out))
    return out


def conv3x3_dgrad(dout, w):
    dout = _f64(dout)
    w = _f64(w)
    N, H, W, Co = dout.shape
    Ci = w.shape[2]
    din = np.empty((N, H, W, Ci))
    lib().orc_conv3x3_dgrad(N, H, W, Ci, Co, _ptr(dout), _ptr(w), _ptr(din))
    return din


def conv3x3_wgrad(x, dout):
    x = _f64(x)
    dout = _f64(dout)
    N, H, W, Ci = x.shape
    Co = dout.shape[3]
    dw = np.empty((3, 3, Ci, Co))
    db = np.empty(Co)
    lib().orc_conv3x3_wgrad(N, H, W, Ci, Co, _ptr(x), _ptr(dout), _ptr(dw), _ptr(db))
    return dw, db
