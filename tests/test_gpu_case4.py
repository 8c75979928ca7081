"""Immersed-boundary leakage (the paper's validation Case IV, Sec. 6.3).

A circular cell under a constant membrane tension (Eq. membraneforce) and no
mass source shrinks because the discrete delta kernel is not divergence-free:
fluid leaks through the membrane.  Refining the lattice by 2 (domain, cell
diameter 10 -> 80 lattice units, T x4, phi_m / 2) the relative area loss
should fall about in proportion to the spacing: the paper reports an order of
convergence of about 1 (0.9891 between its two finest lattices).  Checked
here on the GPU path (FP32 storage, vertices 0.5 lattice units apart, periodic
lattice):
  - the cell loses area at every level (leakage, not growth);
  - the loss falls with every refinement, at an observed order within
    [0.8, 1.5] between each pair of levels and within [0.8, 1.3] between the
    two finest (measured here: 1.34, 1.25, 1.15);
  - the loss is a property of the discretisation, not of the storage: FP64
    storage gives the same loss at the coarsest level to 1e-3 relative.
"""
import math

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


def area_loss(lb, w, precision):
    T = w.tissue
    sim = lb.Simulation(w.params, precision, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.step(1)
    a0 = float(sim.fields(16)["area"][0])
    sim.step(w.n_steps - 1)
    a1 = float(sim.fields(16)["area"][0])
    sim.close()
    return (a0 - a1) / a0


def test_case4_leakage_converges_first_order(lb):
    loss = [area_loss(lb, li.case4(k), lb.LBIB_FP32) for k in range(4)]
    print("relative area loss by level:", ["%.3e" % x for x in loss])
    assert all(x > 0 for x in loss)
    orders = [math.log2(loss[k] / loss[k + 1]) for k in range(3)]
    print("observed orders:", ["%.3f" % o for o in orders])
    assert all(0.8 <= o <= 1.5 for o in orders), orders
    assert 0.8 <= orders[-1] <= 1.3, orders


def test_case4_loss_independent_of_storage(lb):
    w = li.case4(0)
    l32 = area_loss(lb, w, lb.LBIB_FP32)
    l64 = area_loss(lb, w, lb.LBIB_FP64)
    assert abs(l32 - l64) / l64 < 1e-3, (l32, l64)
