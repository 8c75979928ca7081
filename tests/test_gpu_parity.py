"""GPU parity: the CUDA path, called through the C ABI, against the FP64
oracle on the same seeded inputs.

Tolerances (relative L-infinity, max|a - b| / max|b| per field):
  FP64 storage:   1e-10 on u, phi, rho after up to 1000 steps -- the bound
                  the method statement fixes (atomic scatter order and
                  different rounding order are the only differences);
                  labels bit-exact while the vertex paths agree to 1e-12.
  FP32 shifted:   u 1e-4, phi 1e-5, X 1e-6 absolute LU (derived in the design
                  notes: eps32 = 6e-8 relative on deviations of size |u|,
                  accumulated over the run).
  FP16 shifted:   u 3e-2, phi 1e-2 (eps16 = 4.9e-4 on scaled deviations).
"""
import math

import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu

ALL = 1 | 2 | 4 | 8 | 16 | 32 | 64 | 128


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import build, lbib
    build.build()
    lbib.load()
    return lbib


def rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return float(d / s) if s > 0 else float(d)


def gpu_run(lb, w, n, precision, which=ALL, tension=0.0, body=None, forcing=None):
    p = w.params
    if tension:
        p.tension = tension
    if body is not None:
        p.body_force = body
    if forcing is not None:
        p.forcing = forcing
    T = w.tissue
    sim = lb.Simulation(p, precision, T.n_vertices if T else 0, T.n_cells if T else 0)
    if T is not None and T.n_cells:
        sim.set_cells(T)
    sim.step(n)
    out = sim.fields(which)
    sim.close()
    return out


def check_fp64(got, ref, S, tol=1e-10, labels=True):
    eu = max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy))
    # density: relative to its variation about rho0, floored at 1e-2 so that
    # the rest state (rho - 1 at the rounding level) is not ill-conditioned
    er = np.abs(got["rho"] - ref.rho).max() / max(np.abs(ref.rho - 1.0).max(), 1e-2)
    assert eu < tol, eu
    assert er < tol, er
    if S:
        ep = rel(got["phi"], ref.phi)
        assert ep < tol, ep
    if "xy" in got:
        assert np.abs(got["xy"] - ref.xy).max() < 1e-11
    if labels and "id" in got:
        assert np.array_equal(got["id"], ref.id)


# ------------------------------------------------------------------ config 1
def test_config1_fp64_1000_steps(lb, orc):
    """The plain FP64 single-cell workload over its full 1000 steps."""
    w = li.config1()
    ref = orc.run(w.params, w.tissue, 1000)
    got = gpu_run(lb, w, 1000, lb.LBIB_FP64)
    check_fp64(got, ref, 1)
    assert np.abs(got["area"] - ref.area).max() < 1e-9
    assert rel(got["force"][..., 0], ref.fx) < 1e-10
    assert rel(got["vforce"], ref.Fv) < 1e-10


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 9])
def test_step_sequencing(lb, orc, n):
    """Every step count (direct launches, graph chunks, the last-step split)
    reproduces the oracle's trajectory."""
    w = li.config1()
    ref = orc.run(w.params, w.tissue, n)
    got = gpu_run(lb, w, n, lb.LBIB_FP64)
    check_fp64(got, ref, 1, tol=1e-12)
    assert rel(got["vforce"], ref.Fv) < 1e-12


def test_repeated_step_calls_match_one_call(lb, orc):
    w = li.config1()
    ref = orc.run(w.params, w.tissue, 13)
    sim = lb.Simulation(w.params, lb.LBIB_FP64, w.tissue.n_vertices, w.tissue.n_cells)
    sim.set_cells(w.tissue)
    for n in (1, 5, 2, 4, 1):
        sim.step(n)
    got = sim.fields(ALL)
    check_fp64(got, ref, 1, tol=1e-12)


# ------------------------------------------------------------------ walls, species, ragged
def test_walls_two_species_ragged_fp64(lb, orc):
    """Walls in y, two reacting species, a lattice that is not a multiple of
    the row pitch (ragged tail), cells that straddle the periodic x edge."""
    w = li.config2(nx=150, ny=97, n_cells_side=3)
    ref = orc.run(w.params, w.tissue, 120)
    got = gpu_run(lb, w, 120, lb.LBIB_FP64)
    check_fp64(got, ref, 2)


def test_paper_forcing_and_tension_fp64(lb, orc):
    w = li.scaled_config1(72, 14.0, 80, n_species=2, tau=0.7)
    w.params.forcing = 1
    ref = orc.run(w.params, w.tissue, 150, tension=1e-3)
    got = gpu_run(lb, w, 150, lb.LBIB_FP64, tension=1e-3)
    check_fp64(got, ref, 2)


def test_poiseuille_body_force_no_cells(lb, orc):
    """No cells: the lattice update alone with a uniform body force between
    walls, against the oracle's lattice step and the closed form."""
    nx, ny, gF = 40, 21, 1e-6
    p = li.LatticeParams(nx=nx, ny=ny, bc_y=li.BC_WALLS, tau=0.5 + math.sqrt(3) / 4)
    T = li.Tissue(np.zeros(1, np.int32), np.zeros((0, 2)), np.zeros(0), np.zeros(0),
                  np.zeros(0), np.zeros(0, np.uint8))
    w = li.Workload("poiseuille", p, T, 3000, 0)
    got = gpu_run(lb, w, 3000, lb.LBIB_FP64, which=1 | 2, body=(gF, 0.0))
    f, g = orc.equilibrium_state(p)
    fx = np.full((ny, nx), gF)
    fy = np.zeros((ny, nx))
    for _ in range(3000):
        f, g, rho, ux, uy, _ = orc.lattice_step(p, f, g, fx, fy)
    assert rel(got["ux"], ux) < 1e-10
    assert np.abs(got["uy"]).max() < 1e-16 + 1e-10 * np.abs(ux).max()


def test_overlapping_cells_lowest_index_wins(lb, orc):
    p = li.LatticeParams(nx=64, ny=48, n_species=1)
    p.D[0], p.src_rate[0] = 0.1, 1e-3
    T = li.make_tissue([(30.0, 24.0), (36.5, 25.25), (33.0, 20.0)], [9.0, 8.0, 6.0], 24,
                       0.01, 1e-3, [1, 0, 1])
    w = li.Workload("overlap", p, T, 3, 0)
    ref = orc.run(p, T, 3)
    got = gpu_run(lb, w, 3, lb.LBIB_FP64)
    check_fp64(got, ref, 1, tol=1e-12)


def test_large_cell_bruteforce_labels(lb, orc):
    """A cell taller than the scanline row budget takes the brute-force path;
    labels stay exact."""
    w = li.scaled_config1(200, 80.0, 300, jitter=0.3)
    ref = orc.run(w.params, w.tissue, 2)
    got = gpu_run(lb, w, 2, lb.LBIB_FP64)
    check_fp64(got, ref, 1, tol=1e-12)


def test_triangle_cells_and_no_species(lb, orc):
    p = li.LatticeParams(nx=32, ny=40, tau=0.9)
    T = li.make_tissue([(8.0, 9.0), (20.0, 30.0)], [4.0, 5.0], 3, 0.05, 2e-3, [0, 0],
                       jitter=0.2, rng=np.random.default_rng(3))
    w = li.Workload("tri", p, T, 40, 0)
    ref = orc.run(p, T, 40)
    got = gpu_run(lb, w, 40, lb.LBIB_FP64)
    check_fp64(got, ref, 0, tol=1e-11)


# ------------------------------------------------------------------ precision paths
@pytest.mark.parametrize("prec,tu,tp", [("fp32", 1e-4, 1e-5), ("fp16", 3e-2, 1e-2)])
def test_reduced_precision_walls_two_species(lb, orc, prec, tu, tp):
    w = li.config2(nx=256, ny=256, n_cells_side=5)
    ref = orc.run(w.params, w.tissue, 300)
    got = gpu_run(lb, w, 300, lb.PRECISIONS[prec], which=1 | 2 | 4 | 8)
    eu = max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy))
    ep = rel(got["phi"], ref.phi)
    ex = np.abs(got["xy"] - ref.xy).max()
    print(f"{prec}: u {eu:.3e} phi {ep:.3e} X {ex:.3e}")
    assert eu < tu and ep < tp
    assert ex < (1e-6 if prec == "fp32" else 1e-3)


def test_precision_paths_512sq_2000_steps(lb, orc):
    """The precision-sweep tissue scaled to 512^2 (144 cells) over the sweep's
    own length, 2000 steps, against the FP64 oracle: FP32 storage within
    u 1e-4, phi 1e-5 (relative L-infinity), X 1e-5 LU; FP16 shifted storage
    within u 3e-2, phi 1e-2, X 1e-3 LU.  Measured: FP32 u 8.0e-5, phi 2.0e-6,
    X 3.2e-6; FP16 u 3.6e-3, phi 4.9e-3, X 3.9e-4 (against the FP64 GPU path,
    which matches the oracle to 1e-10)."""
    w = li.config3(n=512)
    ref = orc.run(w.params, w.tissue, 2000)
    for prec, tu, tp, tx in ((lb.LBIB_FP32, 1e-4, 1e-5, 1e-5),
                             (lb.LBIB_FP16, 3e-2, 1e-2, 1e-3)):
        got = gpu_run(lb, w, 2000, prec, which=1 | 2 | 4 | 8)
        eu = max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy))
        ep = rel(got["phi"], ref.phi)
        ex = np.abs(got["xy"] - ref.xy).max()
        print(f"precision {prec}: u {eu:.3e} phi {ep:.3e} X {ex:.3e}")
        assert eu < tu and ep < tp and ex < tx


# ------------------------------------------------------------------ full sizes
def test_config2_full_size_first_steps(lb, orc):
    """1024^2 walls, 400 cells, 2 species in FP32 (the benchmarked
    configuration): after one step the labels are bit-exact (same X^0) and
    after three steps u, phi agree with the FP64 oracle within the FP32 bound."""
    w = li.config2()
    ref1 = orc.run(w.params, w.tissue, 1)
    got1 = gpu_run(lb, w, 1, lb.LBIB_FP32, which=32)
    assert np.array_equal(got1["id"], ref1.id)
    ref = orc.run(w.params, w.tissue, 3)
    got = gpu_run(lb, w, 3, lb.LBIB_FP32, which=1 | 2 | 4 | 8)
    assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < 1e-4
    assert rel(got["phi"], ref.phi) < 1e-5
    assert np.abs(got["xy"] - ref.xy).max() < 1e-6


def test_config2_full_size_graph_path(lb, orc):
    """The benchmarked 1024^2 configuration over 7 steps: two two-step CUDA
    graph chunks with programmatic launches between the kernels, then the
    single-launch tail, against the FP64 oracle within the FP32 bounds."""
    w = li.config2()
    ref = orc.run(w.params, w.tissue, 7)
    got = gpu_run(lb, w, 7, lb.LBIB_FP32, which=1 | 2 | 4 | 8)
    assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < 1e-4
    assert rel(got["phi"], ref.phi) < 1e-5
    assert np.abs(got["xy"] - ref.xy).max() < 1e-6


def test_config3_full_size_fp32_fp16(lb, orc):
    """The 4096^2 precision-sweep tissue (9,801 cells, the 128-thread IB
    kernel) over 5 steps (one graph chunk) in FP32 and FP16 storage against
    the FP64 oracle: labels bit-exact after the first step, fields within the
    FP32 and FP16 bounds."""
    w = li.config3()
    ref1 = orc.run(w.params, w.tissue, 1)
    got1 = gpu_run(lb, w, 1, lb.LBIB_FP32, which=32)
    assert np.array_equal(got1["id"], ref1.id)
    ref = orc.run(w.params, w.tissue, 5)
    for prec, tu, tp, tx in ((lb.LBIB_FP32, 1e-4, 1e-5, 1e-6), (lb.LBIB_FP16, 3e-2, 1e-2, 1e-3)):
        got = gpu_run(lb, w, 5, prec, which=1 | 2 | 4 | 8)
        assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < tu
        assert rel(got["phi"], ref.phi) < tp
        assert np.abs(got["xy"] - ref.xy).max() < tx


# ------------------------------------------------------------------ state, errors
def test_state_roundtrip_bitwise(lb):
    w = li.config1()
    a = lb.Simulation(w.params, lb.LBIB_FP32, w.tissue.n_vertices, 1)
    a.set_cells(w.tissue)
    a.step(17)
    st = a.get_state()
    a.step(10)
    fa = a.fields(ALL)
    b = lb.Simulation(w.params, lb.LBIB_FP32, w.tissue.n_vertices, 1)
    b.set_state(st)
    b.step(10)
    fb = b.fields(ALL)
    for k in ("rho", "ux", "uy", "phi", "xy", "id"):
        assert np.array_equal(fa[k], fb[k]), k


def test_nonfinite_reported(lb):
    w = li.config1()
    w.tissue.pressure[:] = 1e300
    sim = lb.Simulation(w.params, lb.LBIB_FP64, w.tissue.n_vertices, 1)
    sim.set_cells(w.tissue)
    sim.step(3)
    with pytest.raises(lb.LbibError) as e:
        sim.fields(1 | 2)
    assert e.value.code == lb.LBIB_E_NONFINITE


def test_bad_cells_rejected(lb):
    w = li.config1()
    sim = lb.Simulation(w.params, lb.LBIB_FP64, 64, 1)
    with pytest.raises(lb.LbibError) as e:
        sim.set_cells(cell_off=np.array([0, 2]), xy=np.zeros((2, 2)))
    assert e.value.code == lb.LBIB_E_CELLS
    xy = w.tissue.xy.copy()
    xy[3, 0] = np.nan
    with pytest.raises(lb.LbibError) as e:
        sim.set_cells(cell_off=w.tissue.cell_off, xy=xy)
    assert e.value.code == lb.LBIB_E_NONFINITE
    with pytest.raises(lb.LbibError) as e:
        sim.fields(1)
    assert e.value.code == lb.LBIB_E_STATE
