"""The asynchronous readback of the cell outputs (lbib_get_cells_async /
lbib_wait_readback) against the synchronous lbib_get_fields().

  - one readback after a step: vertex positions and FP64 areas bit-identical
    to lbib_get_fields(LBIB_X | LBIB_AREA) of the same state;
  - the calls that move the cells wait for a pending readback: positions read
    asynchronously before lbib_step(), lbib_advance() or an ensemble step are
    the ones before the step, bit for bit, although the copy runs after those
    calls return;
  - a pipelined loop (advance one step, wait for the previous step's readback,
    start this step's) returns every step's positions: they match a loop with
    synchronous reads to the atomic-order noise of the spreading (1e-9 LU,
    the bound of the ensemble tests);
  - bad arguments are refused, and destroying a context with a readback in
    flight waits for it.
"""
import ctypes

import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import build, lbib
    build.build()
    lbib.load()
    return lbib


def _pinned(n):
    import torch
    return torch.zeros(n, dtype=torch.float64).pin_memory()


def _sim(lb):
    w = li.config2(nx=200, ny=150, n_cells_side=4)
    sim = lb.Simulation(w.params, lb.LBIB_FP32, w.tissue.n_vertices, w.tissue.n_cells)
    sim.set_cells(w.tissue)
    return w, sim


def test_readback_matches_get_fields(lb):
    w, sim = _sim(lb)
    T = w.tissue
    sim.advance(3)
    xy, area = _pinned(2 * T.n_vertices), _pinned(T.n_cells)
    lb.lbib_get_cells_async(sim.ctx, lb.LBIB_X | lb.LBIB_AREA, xy.data_ptr(), area.data_ptr())
    lb.lbib_wait_readback(sim.ctx)
    ref = sim.fields(lb.LBIB_X | lb.LBIB_AREA)
    assert np.array_equal(xy.numpy().reshape(-1, 2), ref["xy"].reshape(-1, 2))
    assert np.array_equal(area.numpy(), ref["area"])
    lb.lbib_wait_readback(sim.ctx)   # nothing outstanding: OK
    sim.close()


@pytest.mark.parametrize("how", ["step", "advance1", "advance4", "set_cells"])
def test_calls_that_move_cells_wait_for_the_readback(lb, how):
    w, sim = _sim(lb)
    T = w.tissue
    sim.advance(2)
    before = sim.fields(lb.LBIB_X)["xy"].copy()
    xy = _pinned(2 * T.n_vertices)
    lb.lbib_get_cells_async(sim.ctx, lb.LBIB_X, xy.data_ptr(), None)
    if how == "step":
        sim.step(3)
    elif how == "advance1":
        sim.advance(1)
    elif how == "advance4":
        sim.advance(4)
    else:
        sim.set_cells(T)
    lb.lbib_wait_readback(sim.ctx)
    assert np.array_equal(xy.numpy().reshape(-1, 2), before.reshape(-1, 2))
    after = sim.fields(lb.LBIB_X)["xy"]
    if how != "set_cells":
        assert not np.array_equal(after, before)   # the cells did move
    sim.close()


def test_pipelined_loop_returns_every_step(lb):
    n = 6
    w, sim = _sim(lb)
    T = w.tissue
    bufs = [(_pinned(2 * T.n_vertices), _pinned(T.n_cells)) for _ in range(2)]
    got = []
    for k in range(n):
        sim.advance(1)
        if k > 0:
            lb.lbib_wait_readback(sim.ctx)
            got.append((bufs[(k - 1) % 2][0].numpy().copy(), bufs[(k - 1) % 2][1].numpy().copy()))
        xy, area = bufs[k % 2]
        lb.lbib_get_cells_async(sim.ctx, lb.LBIB_X | lb.LBIB_AREA, xy.data_ptr(), area.data_ptr())
    lb.lbib_wait_readback(sim.ctx)
    got.append((bufs[(n - 1) % 2][0].numpy().copy(), bufs[(n - 1) % 2][1].numpy().copy()))
    sim.close()
    w2, ref = _sim(lb)
    for k in range(n):
        ref.advance(1)
        f = ref.fields(lb.LBIB_X | lb.LBIB_AREA)
        assert np.abs(got[k][0].reshape(-1, 2) - f["xy"].reshape(-1, 2)).max() < 1e-9, k
        assert np.abs(got[k][1] - f["area"]).max() < 1e-7, k
    ref.close()


def test_ensemble_step_waits_for_a_tissue_readback(lb):
    ws = li.config4(seed=44, n_tissues=2, n_steps=4, side_min=96, side_max=128)
    ens = lb.Ensemble([w.params for w in ws], [w.tissue for w in ws])
    ens.step(2)
    before = ens.fields(0, lb.LBIB_X)["xy"].copy()
    xy = _pinned(2 * ws[0].tissue.n_vertices)
    lb.lbib_get_cells_async(ens.ctx[0], lb.LBIB_X, xy.data_ptr(), None)
    ens.step(3)
    lb.lbib_wait_readback(ens.ctx[0])
    assert np.array_equal(xy.numpy().reshape(-1, 2), before.reshape(-1, 2))
    ens.close()


def test_readback_arguments_and_destroy(lb):
    w, sim = _sim(lb)
    T = w.tissue
    xy = _pinned(2 * T.n_vertices)
    with pytest.raises(lb.LbibError):
        lb.lbib_get_cells_async(sim.ctx, lb.LBIB_RHO, xy.data_ptr(), None)
    with pytest.raises(lb.LbibError):
        lb.lbib_get_cells_async(sim.ctx, lb.LBIB_X, None, None)
    with pytest.raises(lb.LbibError):
        lb.lbib_get_cells_async(sim.ctx, lb.LBIB_AREA, xy.data_ptr(), None)
    sim.advance(1)
    lb.lbib_get_cells_async(sim.ctx, lb.LBIB_X, xy.data_ptr(), None)
    sim.close()   # waits for the copy in flight
    assert np.isfinite(xy.numpy()).all()
