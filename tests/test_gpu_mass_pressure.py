"""GPU parity of the per-cell mass sources with the area controller
(Sec. 3.2.3; reading c29) and of internal pressure nodes (Sec. 6.1; reading
c30) against the FP64 oracle.

  - one growing cell, constant source, a frame of pressure nodes at the
    periodic seam: FP64 within 1e-10 (velocity, density, positions, areas)
    after 120 steps, through the graphed path (one call) and split calls;
  - walled tissue of 9 cells with per-cell rates, the proportional area
    controller towards per-cell set points and pressure nodes on a column:
    FP64 within 1e-10 after 60 steps; FP32 within the FP32 bounds (u 1e-4,
    X 1e-6 lattice units); FP16 shifted storage within its bounds (u 3e-2,
    X 1e-3);
  - a static per-node source field (random sources and sinks) on top of the
    cells' sources: FP64 within 1e-10, FP32 within its bounds;
  - the set-up calls need contexts created with the feature; ensembles
    refuse the features.
"""
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


def _frame(ny, nx):
    pm = np.zeros((ny, nx), np.uint8)
    pm[0, :] = 1
    pm[:, 0] = 1
    return pm


def _growing_cell():
    n = 64
    p = li.LatticeParams(nx=n, ny=n, tau=1.0, rho0=1.0)
    p.mass_sources, p.pressure_nodes, p.pressure_rho = 1, 1, 1.0
    T = li.make_tissue([(n / 2 + 0.3, n / 2 - 0.2)], [8.0], 64, 0.0, 0.0, [0])
    return p, T, np.array([1e-3]), None, _frame(n, n)


def _tissue():
    w = li.config2(nx=96, ny=80, n_cells_side=3)
    p, T = w.params, w.tissue
    p.mass_sources, p.mass_alpha = 1, 2e-5
    p.pressure_nodes, p.pressure_rho = 1, 1.0
    rng = np.random.default_rng(31)
    rate = 2e-4 * rng.uniform(-1, 1, size=T.n_cells)
    import oracle
    oracle.build()
    area = oracle.cell_areas(T.cell_off, T.xy)
    target = area * rng.uniform(0.8, 1.25, size=T.n_cells)
    pm = np.zeros((p.ny, p.nx), np.uint8)
    pm[:, 0] = 1
    return p, T, rate, target, pm


def _gpu(lb, case, prec, calls):
    p, T, rate, target, pm = case
    sim = lb.Simulation(p, prec, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.set_mass_sources(rate, target)
    sim.set_pressure_nodes(pm)
    for n in calls:
        sim.step(n)
    out = sim.fields(ALL)
    sim.close()
    return out


def _oracle(orc, case, n):
    p, T, rate, target, pm = case
    return orc.run(p, T, n, mass_rate=rate, target_area=target, pmask=pm)


def _check_fp64(got, ref):
    assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < 1e-10
    assert rel(got["rho"], ref.rho) < 1e-12
    assert np.abs(got["xy"] - ref.xy).max() < 1e-10
    assert rel(got["area"], ref.area) < 1e-12
    assert np.array_equal(got["id"], ref.id)


@pytest.mark.parametrize("calls", [(120,), (57, 63)])
def test_growing_cell_fp64(lb, orc, calls):
    case = _growing_cell()
    ref = _oracle(orc, case, 120)
    got = _gpu(lb, case, lb.LBIB_FP64, calls)
    _check_fp64(got, ref)
    assert ref.area[0] > 1.1 * orc.cell_areas(case[1].cell_off, case[1].xy)[0]


@pytest.mark.parametrize("calls", [(60,), (1, 36, 23)])
def test_area_controller_tissue_fp64(lb, orc, calls):
    case = _tissue()
    ref = _oracle(orc, case, 60)
    _check_fp64(_gpu(lb, case, lb.LBIB_FP64, calls), ref)


@pytest.mark.parametrize("prec,tu,tx", [("fp32", 1e-4, 1e-6), ("fp16", 3e-2, 1e-3)])
def test_area_controller_tissue_reduced(lb, orc, prec, tu, tx):
    case = _tissue()
    ref = _oracle(orc, case, 60)
    got = _gpu(lb, case, lb.PRECISIONS[prec], (60,))
    eu = max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy))
    ex = np.abs(got["xy"] - ref.xy).max()
    print(f"{prec}: u {eu:.2e}  X {ex:.2e}")
    assert eu < tu and ex < tx


def _with_node_sources(case):
    p, T, rate, target, pm = case
    p.node_sources = 1
    rng = np.random.default_rng(32)
    ns = 1e-4 * rng.uniform(-1, 1, size=(p.ny, p.nx))
    return p, T, rate, target, pm, ns


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_node_sources_vs_oracle(lb, orc, prec):
    p, T, rate, target, pm, ns = _with_node_sources(_tissue())
    ref = orc.run(p, T, 60, mass_rate=rate, target_area=target, pmask=pm, node_source=ns)
    sim = lb.Simulation(p, lb.PRECISIONS[prec], T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.set_mass_sources(rate, target)
    sim.set_pressure_nodes(pm)
    sim.set_node_sources(ns)
    sim.step(60)
    got = sim.fields(ALL)
    sim.close()
    if prec == "fp64":
        _check_fp64(got, ref)
    else:
        assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < 1e-4
        assert np.abs(got["xy"] - ref.xy).max() < 1e-6


def test_setup_calls_need_the_feature(lb):
    w = li.config2(nx=96, ny=80, n_cells_side=3)
    T = w.tissue
    sim = lb.Simulation(w.params, lb.LBIB_FP32, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    with pytest.raises(lb.LbibError):
        sim.set_mass_sources(np.zeros(T.n_cells))
    with pytest.raises(lb.LbibError):
        sim.set_pressure_nodes(np.zeros((w.params.ny, w.params.nx), np.uint8))
    with pytest.raises(lb.LbibError):
        sim.set_node_sources(np.zeros((w.params.ny, w.params.nx)))
    sim.close()
    for field in ("mass_sources", "pressure_nodes", "node_sources"):
        p = li.config2(nx=96, ny=80, n_cells_side=3).params
        setattr(p, field, 1)
        with pytest.raises(lb.LbibError):
            lb.Ensemble([p], [T])
