"""Seeded synthetic tissue inputs for the LBIBCell coupled step.

This module is shared by the FP64 oracle, the CUDA path, the tests and the
bench.  It builds the *problem* (lattice parameters, cell polygons, per-edge
spring data, per-cell pressure and source flags) and nothing of the method:
no lattice Boltzmann, immersed-boundary or force arithmetic lives here.

Geometry conventions (both solvers share them):
  * lattice node (i, j) sits at position (i, j); x (index i) is fastest;
  * cells are closed polygons stored CSR-style: the vertices of cell c are
    rows cell_off[c] .. cell_off[c+1]-1 of ``xy`` (float64, shape (V, 2)),
    counter-clockwise (Sec. 3.1, Fig. 2 of the paper: polygons are CCW);
  * edge l joins vertex l to the next vertex of the same cell (cyclic);
    ``rest_len[l]`` and ``k_spring[l]`` belong to that edge;
  * ``src_flag[c]`` bit s marks cell c as a source of species s.

Workload recipes follow the five configurations the method is measured on
(plain FP64 single cell; 1024^2 walls with 400 hexagonally packed cells and a
two-species linear reaction; 4096^2 precision sweep with 10,000 cells;
a 64-tissue ensemble; 256^2 steady morphogen solves on random hexagonal
tissues).  Every choice the configurations leave open is fixed here and
listed with its reason in the design notes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# bc_y values
BC_PERIODIC = 0
BC_WALLS = 1


@dataclasses.dataclass
class LatticeParams:
    nx: int
    ny: int
    bc_y: int = BC_PERIODIC
    tau: float = 1.0
    rho0: float = 1.0
    n_species: int = 0
    D: List[float] = dataclasses.field(default_factory=lambda: [0.0] * 4)
    decay: List[float] = dataclasses.field(default_factory=lambda: [0.0] * 4)
    # react[a][b]: linear coupling of species b into the rate of species a
    react: List[List[float]] = dataclasses.field(
        default_factory=lambda: [[0.0] * 4 for _ in range(4)])
    src_rate: List[float] = dataclasses.field(default_factory=lambda: [0.0] * 4)
    forcing: int = 0          # 0 = Guo forcing, 1 = the paper's simple term
    fp16_scale: float = 2.0 ** -10
    tension: float = 0.0      # constant membrane tension phi_m (Eq. membraneforce)
    # reaction model: 0 linear (react, decay); 1 Schnakenberg on species 0
    # (receptor R) and 1 (ligand L) with schnak = (gamma, a, b)
    reaction: int = 0
    schnak: List[float] = dataclasses.field(default_factory=lambda: [0.0, 0.0, 0.0])
    noflux: int = 0           # bit s: species s confined to its domain
    # membrane no-flux scheme of the confined species: 0 the equilibrium
    # closure of Sec. 6.1, 1 half-way bounce-back (an option, not the paper's)
    noflux_scheme: int = 0
    # cell junctions (Eq. celljunctionforce): spring constant, rest length,
    # cutoff, renewal period in steps (0 = none)
    junction_k: float = 0.0
    junction_l0: float = 0.0
    junction_lmax: float = 0.0
    junction_period: int = 0
    # mass sources per cell (Sec. 3.2.3): 1 = on (rates and target areas are
    # given per cell), with the area controller gain alpha
    mass_sources: int = 0
    mass_alpha: float = 0.0
    # internal pressure nodes (Sec. 6.1): 1 = a static node mask is given,
    # held at density pressure_rho
    pressure_nodes: int = 0
    pressure_rho: float = 1.0
    # a static mass source per node (the field S(x,t) of Fig. 1): 1 = on
    node_sources: int = 0
    # a mass source mass_beta * phi_s inside the cells (s = mass_species)
    mass_beta: float = 0.0
    mass_species: int = 0
    # 1 = the confined species (noflux) follow the cells' labels of each step
    noflux_dynamic: int = 0


@dataclasses.dataclass
class Tissue:
    cell_off: np.ndarray      # int32 (C+1,)
    xy: np.ndarray            # float64 (V, 2)
    rest_len: np.ndarray      # float64 (V,)  edge l -> next
    k_spring: np.ndarray      # float64 (V,)
    pressure: np.ndarray      # float64 (C,)
    src_flag: np.ndarray      # uint8 (C,)

    @property
    def n_cells(self) -> int:
        return int(self.cell_off.shape[0] - 1)

    @property
    def n_vertices(self) -> int:
        return int(self.xy.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    params: LatticeParams
    tissue: Tissue
    n_steps: int
    seed: int


def _next_index(cell_off: np.ndarray) -> np.ndarray:
    """Index of the next vertex of the same cell for every vertex."""
    V = int(cell_off[-1])
    nxt = np.arange(1, V + 1, dtype=np.int64)
    for c in range(cell_off.shape[0] - 1):
        nxt[cell_off[c + 1] - 1] = cell_off[c]
    return nxt


def edge_lengths(cell_off: np.ndarray, xy: np.ndarray) -> np.ndarray:
    """Length of edge l -> next(l); used to set rest lengths to the initial
    edge lengths, which is part of the problem statement, not the method."""
    nxt = _next_index(cell_off)
    d = xy[nxt] - xy
    return np.hypot(d[:, 0], d[:, 1])


def polygon_ring(cx: float, cy: float, radius: float, n: int) -> np.ndarray:
    """n vertices of a regular CCW polygon on a circle."""
    a = 2.0 * math.pi * np.arange(n) / n
    return np.stack([cx + radius * np.cos(a), cy + radius * np.sin(a)], axis=1)


def make_tissue(centres, radii, n_vert, k, pressure, src_flag, jitter=0.0,
                rng: Optional[np.random.Generator] = None) -> Tissue:
    """Polygons on circles, optional uniform per-coordinate vertex jitter,
    rest lengths taken after the jitter."""
    rings = [polygon_ring(cx, cy, r, n_vert) for (cx, cy), r in zip(centres, radii)]
    xy = np.concatenate(rings, axis=0).astype(np.float64)
    if jitter:
        xy = xy + rng.uniform(-jitter, jitter, size=xy.shape)
    C = len(rings)
    off = (np.arange(C + 1) * n_vert).astype(np.int32)
    L0 = edge_lengths(off, xy)
    ks = np.broadcast_to(np.asarray(k, dtype=np.float64), (C,))
    kv = np.repeat(ks, n_vert).astype(np.float64)
    pv = np.broadcast_to(np.asarray(pressure, dtype=np.float64), (C,)).copy()
    return Tissue(off, np.ascontiguousarray(xy), L0, kv, pv,
                  np.asarray(src_flag, dtype=np.uint8).copy())


# ---------------------------------------------------------------------------
# the five measured configurations
# ---------------------------------------------------------------------------

def config1(seed: int = 1, n_steps: int = 1000) -> Workload:
    """Plain method, FP64: 64x64 periodic, tau 1, one 64-vertex cell of
    radius 12 at the domain centre, +-0.5 uniform vertex jitter, springs
    k=0.01 with rest length = jittered edge length, pressure 1e-3, one
    species D=0.1 with source 1e-3 inside the cell and decay 1e-3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = LatticeParams(nx=64, ny=64, bc_y=BC_PERIODIC, tau=1.0, rho0=1.0, n_species=1)
    P.D[0] = 0.1
    P.decay[0] = 1e-3
    P.src_rate[0] = 1e-3
    T = make_tissue([(32.0, 32.0)], [12.0], 64, 0.01, 1e-3, [1], jitter=0.5, rng=rng)
    return Workload("c1_64x64_fp64_1cell", P, T, n_steps, seed)


def hex_centres_1024():
    """20 x 20 hexagonal packing on 1024^2: spacing 51.2 in x, row pitch
    51.2*sqrt(3)/2, odd rows shifted by half a spacing, rows centred in y."""
    a = 51.2
    h = a * math.sqrt(3.0) / 2.0
    y0 = (1024.0 - 19 * h) / 2.0
    cs = []
    for j in range(20):
        for i in range(20):
            cs.append((a * i + a / 2 + (a / 2 if j % 2 else 0.0), y0 + j * h))
    return cs


def config2(seed: int = 2, n_steps: int = 5000, nx: int = 1024, ny: int = 1024,
            n_cells_side: int = 20) -> Workload:
    """FP32 lattice, FP64 vertices: 1024^2, no-slip walls in y, periodic x,
    tau 0.8; 400 cells of 100 vertices, radius 20 with per-cell +-10% noise,
    springs k=0.02, pressure 1e-3; two species a, b with
    a_t = 0.05a - 0.1b + s, b_t = 0.1a - 0.15b, D_a=0.05, D_b=0.1, source
    s=1e-3 into a in a seeded 10% of the cells.  ``nx, ny, n_cells_side``
    scale the same recipe down for tests (spacing nx/n_cells_side)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = LatticeParams(nx=nx, ny=ny, bc_y=BC_WALLS, tau=0.8, rho0=1.0, n_species=2)
    P.D[0], P.D[1] = 0.05, 0.1
    P.react[0][0], P.react[0][1] = 0.05, -0.1
    P.react[1][0], P.react[1][1] = 0.1, -0.15
    P.src_rate[0] = 1e-3
    a = nx / n_cells_side
    h = a * math.sqrt(3.0) / 2.0
    y0 = (ny - (n_cells_side - 1) * h) / 2.0
    centres = [(a * i + a / 2 + (a / 2 if j % 2 else 0.0), y0 + j * h)
               for j in range(n_cells_side) for i in range(n_cells_side)]
    C = len(centres)
    r_base = 20.0 * a / 51.2
    radii = r_base * (1.0 + rng.uniform(-0.1, 0.1, size=C))
    n_src = max(1, int(round(0.1 * C)))
    src = np.zeros(C, np.uint8)
    src[rng.choice(C, size=n_src, replace=False)] = 1
    T = make_tissue(centres, radii, 100, 0.02, 1e-3, src)
    w = Workload(f"c2_{nx}x{ny}_fp32_walls_{C}cells_2species", P, T, n_steps, seed)
    w.radii = radii
    return w


def config2_junctions(seed: int = 2, n_steps: int = 5000, period: int = 10) -> Workload:
    """The 1024^2 walled tissue of ``config2`` with cell junctions
    (Eq. celljunctionforce): neighbouring membranes lie about 11 lattice
    units apart (pitch 51.2, radii 20 +- 10%), junctions with k_j = 0.02,
    l_0 = 8 and l_max = 14, renewed every ``period`` steps."""
    w = config2(seed=seed, n_steps=n_steps)
    p = w.params
    p.junction_k, p.junction_l0, p.junction_lmax, p.junction_period = 0.02, 8.0, 14.0, period
    return Workload(w.name.replace("c2_", "c2j_") + f"_junctions_every{period}", p, w.tissue,
                    n_steps, seed)


def config2_growth(seed: int = 2, n_steps: int = 5000, growth: float = 1.2,
                   alpha: float = 2e-6) -> Workload:
    """The 1024^2 walled tissue of ``config2`` growing under the proportional
    area controller (Sec. 3.2.3): every cell's set point is ``growth`` times
    its initial polygon area (regular 100-gon), gain alpha; the rows next to
    the two walls are internal pressure nodes at rho0 that take up the added
    mass."""
    w = config2(seed=seed, n_steps=n_steps)
    p = w.params
    p.mass_sources, p.mass_alpha = 1, alpha
    p.pressure_nodes, p.pressure_rho = 1, 1.0
    n = 100
    poly_area = 0.5 * n * np.asarray(w.radii) ** 2 * math.sin(2.0 * math.pi / n)
    w.mass_rate = np.zeros(w.tissue.n_cells)
    w.target_area = growth * poly_area
    w.pressure_mask = np.zeros((p.ny, p.nx), np.uint8)
    w.pressure_mask[0, :] = 1
    w.pressure_mask[-1, :] = 1
    w.name = w.name.replace("c2_", "c2g_") + f"_area_controller_x{growth:g}"
    return w


def jittered_grid_tissue(rng, nx, ny, spacing, radius, n_vert, k, pressure,
                         centre_jitter, src_fraction, radius_noise=0.0):
    nxc = int(nx // spacing)
    nyc = int(ny // spacing)
    sx = nx / nxc
    sy = ny / nyc
    centres = []
    for j in range(nyc):
        for i in range(nxc):
            centres.append((sx * (i + 0.5), sy * (j + 0.5)))
    C = len(centres)
    cj = rng.uniform(-centre_jitter, centre_jitter, size=(C, 2))
    centres = [(x + dx, y + dy) for (x, y), (dx, dy) in zip(centres, cj)]
    radii = radius * (1.0 + rng.uniform(-radius_noise, radius_noise, size=C)) \
        if radius_noise else np.full(C, radius)
    n_src = max(1, int(round(src_fraction * C)))
    src = np.zeros(C, np.uint8)
    src[rng.choice(C, size=n_src, replace=False)] = 1
    return make_tissue(centres, radii, n_vert, k, pressure, src)


def config3(seed: int = 3, n_steps: int = 2000, n: int = 4096) -> Workload:
    """Precision sweep: n^2 periodic (4096 by default), tau 0.6, cells of 64
    vertices, radius 15, on a jittered grid of spacing n/100 (+-5 LU centre
    jitter), springs k=0.01, pressure 1e-3, one species D=0.1, decay 1e-3,
    source 1e-3 in a seeded 10% of the cells."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = LatticeParams(nx=n, ny=n, bc_y=BC_PERIODIC, tau=0.6, rho0=1.0, n_species=1)
    P.D[0] = 0.1
    P.decay[0] = 1e-3
    P.src_rate[0] = 1e-3
    spacing = 40.96
    T = jittered_grid_tissue(rng, n, n, spacing, 15.0, 64, 0.01, 1e-3, 5.0, 0.1)
    return Workload(f"c3_{n}x{n}_{T.n_cells}cells", P, T, n_steps, seed)


def config4(seed: int = 4, n_tissues: int = 64, n_steps: int = 2000,
            side_min: int = 128, side_max: int = 1024) -> List[Workload]:
    """Ensemble of independent periodic tissues: side = round(sqrt(A)) with A
    log-uniform on [side_min^2, side_max^2]; cells of 64 vertices, radius 15
    on a jittered grid of spacing 40 (about one cell per 1600 nodes);
    k ~ U(0.005, 0.05), tau ~ U(0.6, 1.2); one species as in config 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for t in range(n_tissues):
        A = math.exp(rng.uniform(math.log(side_min ** 2), math.log(side_max ** 2)))
        side = int(round(math.sqrt(A)))
        tau = float(rng.uniform(0.6, 1.2))
        k = float(rng.uniform(0.005, 0.05))
        P = LatticeParams(nx=side, ny=side, bc_y=BC_PERIODIC, tau=tau, rho0=1.0, n_species=1)
        P.D[0] = 0.1
        P.decay[0] = 1e-3
        P.src_rate[0] = 1e-3
        T = jittered_grid_tissue(rng, side, side, 40.0, 15.0, 64, k, 1e-3, 2.0, 0.1)
        out.append(Workload(f"c4_t{t}_{side}", P, T, n_steps, seed))
    return out


def steady_tissue(seed: int, n: int = 256, n_vert: int = 32):
    """Random hexagonal tissue for the steady morphogen solve: 30-80 polygons
    on an n^2 periodic lattice, D ~ U(0.05, 0.2), decay ~ U(1e-4, 1e-2),
    sources in a seeded 5-20% of the cells with rate 1e-3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_target = int(rng.integers(30, 81))
    # hexagonal lattice of pitch a with about n_target sites on n^2
    a = math.sqrt(2.0 * n * n / (math.sqrt(3.0) * n_target))
    h = a * math.sqrt(3.0) / 2.0
    cols = max(1, int(round(n / a)))
    rows = max(1, int(round(n / h)))
    ax = n / cols
    hy = n / rows
    sites = []
    for j in range(rows):
        for i in range(cols):
            sites.append((ax * (i + 0.5) + (ax / 2 if j % 2 else 0.0), hy * (j + 0.5)))
    order = rng.permutation(len(sites))[: min(n_target, len(sites))]
    order.sort()
    centres = [sites[i] for i in order]
    C = len(centres)
    r = 0.42 * min(ax, hy)
    radii = r * (1.0 + rng.uniform(-0.1, 0.1, size=C))
    jit = rng.uniform(-0.05 * r, 0.05 * r, size=(C, 2))
    centres = [(x + dx, y + dy) for (x, y), (dx, dy) in zip(centres, jit)]
    frac = rng.uniform(0.05, 0.20)
    n_src = max(1, int(round(frac * C)))
    src = np.zeros(C, np.uint8)
    src[rng.choice(C, size=n_src, replace=False)] = 1
    T = make_tissue(centres, radii, n_vert, 0.0, 0.0, src)
    P = LatticeParams(nx=n, ny=n, bc_y=BC_PERIODIC, tau=1.0, rho0=1.0, n_species=1)
    P.D[0] = float(rng.uniform(0.05, 0.2))
    P.decay[0] = float(rng.uniform(1e-4, 1e-2))
    P.src_rate[0] = 1e-3
    return P, T


def scaled_config1(n: int, R: float, n_vert: int, seed: int = 11, n_steps: int = 50,
                   jitter: float = 0.5, walls: bool = False, n_species: int = 1,
                   tau: float = 1.0) -> Workload:
    """Config-1 recipe on an n^2 lattice with a cell of radius R (tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = LatticeParams(nx=n, ny=n, bc_y=BC_WALLS if walls else BC_PERIODIC, tau=tau,
                      rho0=1.0, n_species=n_species)
    for s in range(n_species):
        P.D[s] = 0.1 + 0.05 * s
        P.decay[s] = 1e-3
        P.src_rate[s] = 1e-3
    T = make_tissue([(n / 2, n / 2)], [R], n_vert, 0.01, 1e-3, [(1 << n_species) - 1],
                    jitter=jitter, rng=rng)
    return Workload(f"c1s_{n}", P, T, n_steps, seed)


def case4(level: int, max_length: float = 0.5) -> Workload:
    """The immersed-boundary leakage study (validation Case IV, Sec. 6.3): a
    circular cell under the constant membrane tension of Eq. membraneforce,
    no mass source, tau 1, no species.  Level k refines the lattice by 2^k:
    domain 100*2^k, cell diameter 10*2^k lattice units (the DIA values of the
    study's figure), T = 1e4*4^k steps and phi_m = 1e-3/2^k in LB units (the
    study's table: dt ~ dx^2, F^LB ~ dx).  Vertices are max_length lattice
    units apart (the study's MAXLENGTH); the lattice is periodic in place of
    the study's outflow boundary."""
    N = 100 * 2 ** level
    D = 10.0 * 2 ** level
    P = LatticeParams(nx=N, ny=N, bc_y=BC_PERIODIC, tau=1.0, rho0=1.0, n_species=0)
    P.tension = 1e-3 / 2 ** level
    n_vert = int(math.ceil(math.pi * D / max_length))
    T = make_tissue([(N / 2.0, N / 2.0)], [D / 2.0], n_vert, 0.0, 0.0, [0])
    return Workload(f"case4_level{level}_{N}x{N}_dia{int(D)}", P, T, 10000 * 4 ** level, 0)


def case1(level: int, max_length: float = 0.5) -> Workload:
    """Validation Case I (Sec. 6.3): a circular cell grown by a constant point
    mass source at its centre node, no membrane force, tau 1, no species.
    Level k: domain 100*2^k, diameter 10*2^k lattice units, T = 1e4*4^k steps,
    source 1e-2 per step (the study's table: S^LB = S^ND dt/dx^2 with
    S^ND = 1), so that A(T) = A0 + 1e-2 T = A0 (1 + 4/pi).  Pressure nodes at
    rho0 on the periodic seam take up the excess mass, in place of the
    study's iso-pressure outflow boundary."""
    N = 100 * 2 ** level
    D = 10.0 * 2 ** level
    steps = 10000 * 4 ** level
    P = LatticeParams(nx=N, ny=N, bc_y=BC_PERIODIC, tau=1.0, rho0=1.0, n_species=0)
    P.node_sources = 1
    P.pressure_nodes, P.pressure_rho = 1, 1.0
    n_vert = int(math.ceil(math.pi * D / max_length))
    T = make_tissue([(N / 2.0, N / 2.0)], [D / 2.0], n_vert, 0.0, 0.0, [0])
    w = Workload(f"case1_level{level}_{N}x{N}_dia{int(D)}", P, T, steps, 0)
    w.node_source = np.zeros((N, N))
    w.node_source[N // 2, N // 2] = 1e-2
    w.pressure_mask = np.zeros((N, N), np.uint8)
    w.pressure_mask[0, :] = 1
    w.pressure_mask[:, 0] = 1
    return w


def case3(level: int, max_length: float = 0.5) -> Workload:
    """Validation Case III (Sec. 6.3): a circular cell holding one species
    (concentration 1 at the nodes strictly inside the circle, 0 elsewhere,
    no production or decay) that the moving membrane confines, and a mass
    source beta * C at every node inside the cell.  Level k: domain 100*2^k,
    diameter 10*2^k lattice units, T = 1e4*4^k steps, tau = tau_D = 1 (the
    study's table), beta = 1 / T (the study's strength 1 C in its time
    unit), so that the area grows linearly, A(T) = A0 + beta M T with M the
    conserved species mass.  Pressure nodes at rho0 on the periodic seam take
    up the excess mass, in place of the study's outflow boundary."""
    N = 100 * 2 ** level
    D = 10.0 * 2 ** level
    steps = 10000 * 4 ** level
    P = LatticeParams(nx=N, ny=N, bc_y=BC_PERIODIC, tau=1.0, rho0=1.0, n_species=1)
    P.D[0] = 1.0 / 6.0
    P.noflux, P.noflux_dynamic = 1, 1
    P.mass_beta, P.mass_species = 1.0 / steps, 0
    P.pressure_nodes, P.pressure_rho = 1, 1.0
    n_vert = int(math.ceil(math.pi * D / max_length))
    T = make_tissue([(N / 2.0, N / 2.0)], [D / 2.0], n_vert, 0.0, 0.0, [0])
    w = Workload(f"case3_level{level}_{N}x{N}_dia{int(D)}", P, T, steps, 0)
    X, Y = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64))
    inside = np.hypot(X - N / 2.0, Y - N / 2.0) <= D / 2.0 - 0.1
    w.phi0 = inside.astype(np.float64)[None]
    w.pressure_mask = np.zeros((N, N), np.uint8)
    w.pressure_mask[0, :] = 1
    w.pressure_mask[:, 0] = 1
    return w


def case2(level: int, max_length: float = 0.5) -> Workload:
    """Validation Case II (Sec. 6.3): a circular cell grown by a constant mass
    source, uniform over the nodes inside it, no membrane force, tau 1, no
    species.  Level k: domain 100*2^k, diameter 10*2^k lattice units,
    T = 1e4*4^k steps (the study's table), per-node source ln 2 / T so that
    the area doubles by T.  The excess mass leaves through internal pressure
    nodes at rho0 on the periodic seam (row 0 and column 0), in place of the
    study's iso-pressure outflow boundary."""
    N = 100 * 2 ** level
    D = 10.0 * 2 ** level
    steps = 10000 * 4 ** level
    P = LatticeParams(nx=N, ny=N, bc_y=BC_PERIODIC, tau=1.0, rho0=1.0, n_species=0)
    P.mass_sources = 1
    P.pressure_nodes, P.pressure_rho = 1, 1.0
    n_vert = int(math.ceil(math.pi * D / max_length))
    T = make_tissue([(N / 2.0, N / 2.0)], [D / 2.0], n_vert, 0.0, 0.0, [0])
    w = Workload(f"case2_level{level}_{N}x{N}_dia{int(D)}", P, T, steps, 0)
    w.mass_rate = np.array([math.log(2.0) / steps])
    w.pressure_mask = np.zeros((N, N), np.uint8)
    w.pressure_mask[0, :] = 1
    w.pressure_mask[:, 0] = 1
    return w


def voronoi_domains(nx: int, ny: int, spacing: float, seed: int) -> np.ndarray:
    """A static cellular domain: the periodic Voronoi tiling of a jittered
    grid of centres (spacing lattice units, +-spacing/4 jitter); label of a
    node = index of its nearest centre (int32, shape (ny, nx))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gx, gy = max(1, int(round(nx / spacing))), max(1, int(round(ny / spacing)))
    sx, sy = nx / gx, ny / gy
    cx = (np.arange(gx)[None, :] + 0.5) * sx + rng.uniform(-sx / 4, sx / 4, size=(gy, gx))
    cy = (np.arange(gy)[:, None] + 0.5) * sy + rng.uniform(-sy / 4, sy / 4, size=(gy, gx))
    X, Y = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))
    ci = np.floor(X / sx).astype(np.int64)
    cj = np.floor(Y / sy).astype(np.int64)
    best = np.full((ny, nx), np.inf)
    lab = np.zeros((ny, nx), np.int32)
    for dj in (-1, 0, 1):       # the nearest centre lies in a neighbouring grid cell
        for di in (-1, 0, 1):
            i2, j2 = (ci + di) % gx, (cj + dj) % gy
            dx = X - cx[j2, i2]
            dy = Y - cy[j2, i2]
            dx -= nx * np.round(dx / nx)
            dy -= ny * np.round(dy / ny)
            d2 = dx * dx + dy * dy
            m = d2 < best
            best[m] = d2[m]
            lab[m] = (j2 * gx + i2)[m].astype(np.int32)
    return lab


def turing(seed: int = 6, n: int = 1024, n_steps: int = 2000) -> Workload:
    """The Turing example on a static cellular domain (Sec. 4.2, Fig. 5C):
    n^2 periodic lattice at rest (tau 1), receptor R (species 0, D = 0.05,
    confined to its cell) and ligand L (species 1, D = 0.4, free) with the
    Schnakenberg rates gamma = 0.02, a = 0.1, b = 0.9 in LB units, cells of a
    periodic Voronoi tiling of spacing n/20 (400 cells at 1024^2), starting
    from the homogeneous state with +-5 % seeded noise.  Attributes domains
    (labels) and phi0 (initial fields) ride on the workload."""
    P = LatticeParams(nx=n, ny=n, bc_y=BC_PERIODIC, tau=1.0, rho0=1.0, n_species=2)
    P.D[0], P.D[1] = 0.05, 0.4
    P.reaction = 1
    P.schnak = [0.02, 0.1, 0.9]
    P.noflux = 1
    T = Tissue(np.zeros(1, np.int32), np.zeros((0, 2)), np.zeros(0), np.zeros(0),
               np.zeros(0), np.zeros(0, np.uint8))
    w = Workload(f"turing_{n}x{n}_static_voronoi", P, T, n_steps, seed)
    w.domains = voronoi_domains(n, n, n / 20.0, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    a, b = P.schnak[1], P.schnak[2]
    w.phi0 = np.stack([(a + b) * (1 + 0.05 * rng.uniform(-1, 1, size=(n, n))),
                       b / (a + b) ** 2 * (1 + 0.05 * rng.uniform(-1, 1, size=(n, n)))])
    return w


def random_fields(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-scale, scale, size=shape)


def nop_init_params(seed: int, shapes) -> np.ndarray:
    """Initial parameters of the neural operator for the given layer list
    [(name, Ci, Co), ...]: He-normal weights (std sqrt(2 / (9 Ci)); a tenth of
    that for the output layer), zero biases, in the flat layout weights
    (3, 3, Ci, Co) then bias (Co,) per layer.  FP32-representable values."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for name, ci, co in shapes:
        std = math.sqrt(2.0 / (9 * ci)) * (0.1 if name == "out" else 1.0)
        out.append(rng.normal(0.0, std, size=9 * ci * co))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32).astype(np.float64)
