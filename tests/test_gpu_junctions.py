"""GPU parity of the cell junctions (Eq. celljunctionforce, Sec. 3.2.4;
renewal and partner rule: reading c28) against the FP64 oracle.

The partner search runs on the GPU through a grid of vertex bins with the
definition's FP64 operations, so with FP64 storage the partners, and with
them the whole coupled trajectory, match the oracle:
  - walled tissue (hexagonal cells 7 lattice units apart, l_max 8, renewal
    every 5 steps): velocity, concentrations, positions and the vertex
    forces of the output step within 1e-10 after 40 steps, also when the 40
    steps are split over two calls (the renewal count carries over);
  - periodic tissue (jittered grid, pairs across the periodic seam): the
    same bound after 30 steps;
  - FP32 storage within the FP32 bounds (u 1e-4, X 1e-6 lattice units);
  - the junctions change the trajectory (positions move by more than 1e-4
    against a run without them);
  - the profiled step takes the same steps; ensembles refuse junctions.
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


def _walled():
    w = li.config2(nx=96, ny=80, n_cells_side=3)
    p = w.params
    p.junction_k, p.junction_l0, p.junction_lmax, p.junction_period = 0.01, 6.0, 8.0, 5
    return w


def _periodic():
    w = li.config3(n=256)
    p = w.params
    p.junction_k, p.junction_l0, p.junction_lmax, p.junction_period = 0.02, 9.0, 12.0, 4
    return w


def _gpu(lb, w, prec, calls):
    T = w.tissue
    sim = lb.Simulation(w.params, prec, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    for n in calls:
        sim.step(n)
    out = sim.fields(ALL)
    sim.close()
    return out


def _check_fp64(got, ref):
    assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < 1e-10
    assert rel(got["phi"], ref.phi) < 1e-10
    assert np.abs(got["xy"] - ref.xy).max() < 1e-10
    assert rel(got["vforce"], ref.Fv) < 1e-10
    assert np.array_equal(got["id"], ref.id)


@pytest.mark.parametrize("calls", [(40,), (17, 23)])
def test_junctions_walled_fp64(lb, orc, calls):
    w = _walled()
    ref = orc.run(w.params, w.tissue, 40)
    _check_fp64(_gpu(lb, w, lb.LBIB_FP64, calls), ref)


def test_junctions_periodic_fp64(lb, orc):
    w = _periodic()
    ref = orc.run(w.params, w.tissue, 30)
    _check_fp64(_gpu(lb, w, lb.LBIB_FP64, (30,)), ref)


def test_junctions_dense_membranes_fp64(lb, orc):
    """Cells of 400 vertices (0.2 lattice units apart) put well over a hundred
    vertices into one search bin; the partners and the trajectory still follow
    the oracle's brute-force search."""
    w = _walled()
    base = w.tissue
    C = base.n_cells
    n0 = int(base.cell_off[1] - base.cell_off[0])
    centres = [tuple(base.xy[base.cell_off[c]:base.cell_off[c + 1]].mean(axis=0))
               for c in range(C)]
    radii = [float(np.hypot(*(base.xy[base.cell_off[c]] - centres[c]))) for c in range(C)]
    assert n0 == 100
    T = li.make_tissue(centres, radii, 400, 0.02, 1e-3, base.src_flag)
    w.tissue = T
    ref = orc.run(w.params, T, 12)
    _check_fp64(_gpu(lb, w, lb.LBIB_FP64, (12,)), ref)
    p = w.params
    part = orc.junction_partners(p.nx, p.ny, p.bc_y, T.cell_off, ref.xy, p.junction_lmax)
    assert (part >= 0).sum() > 1000


def test_junctions_fp32(lb, orc):
    w = _walled()
    ref = orc.run(w.params, w.tissue, 40)
    got = _gpu(lb, w, lb.LBIB_FP32, (40,))
    assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < 1e-4
    assert np.abs(got["xy"] - ref.xy).max() < 1e-6


def test_junctions_change_the_trajectory(lb):
    w = _walled()
    a = _gpu(lb, w, lb.LBIB_FP64, (40,))
    w.params.junction_period = 0
    b = _gpu(lb, w, lb.LBIB_FP64, (40,))
    assert np.abs(a["xy"] - b["xy"]).max() > 1e-4


def test_junctions_profiled_step_matches(lb):
    """The profiled step takes the same steps: split 25 + 15 over a plain and
    a profiled call, the state equals the plain 40-step run (to 1e-12: the
    spreading's atomic order is not fixed)."""
    w = _walled()
    ref = _gpu(lb, w, lb.LBIB_FP64, (40,))
    T = w.tissue
    sim = lb.Simulation(w.params, lb.LBIB_FP64, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.step(25)
    lat_ms, ib_ms = sim.step_profiled(15)
    got = sim.fields(ALL)
    sim.close()
    assert lat_ms > 0 and ib_ms > 0
    for k in ("ux", "uy", "phi", "vforce"):
        assert rel(got[k], ref[k]) < 1e-12, k
    assert np.abs(got["xy"] - ref["xy"]).max() < 1e-12


def test_junctions_refused_by_ensembles(lb):
    w = _walled()
    with pytest.raises(lb.LbibError):
        lb.Ensemble([w.params], [w.tissue])
