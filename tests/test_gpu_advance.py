"""lbib_advance: the steps of lbib_step without the output work of the last
one.  A context advanced by lbib_advance(n) and then one lbib_step must hold
the state of a context advanced by lbib_step(n + 1): the same kernels and
arithmetic, only the atomic order of the spreading differs (FP64: relative
L-infinity 1e-12 on u and phi, 1e-12 LU on X; FP32: the ensemble-against-
single-tissue tolerance 1e-5 and 1e-9 LU).  Both parities of the step count
are covered (an odd count starts with a direct launch, an even one ends with
the final two-step graph).  Between the two calls only positions and areas
can be read; the lattice fields are refused with LBIB_E_STATE.
"""
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


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("prec,tol,tol_x", [("fp64", 1e-12, 1e-12), ("fp32", 1e-5, 1e-9)])
@pytest.mark.parametrize("n", [1, 6, 7])
def test_advance_then_step_matches_step(lb, prec, tol, tol_x, n):
    w = li.config1() if prec == "fp64" else li.config2(nx=128, ny=128, n_cells_side=2)
    p, T = w.params, w.tissue
    P = lb.PRECISIONS[prec]
    a = lb.Simulation(p, P, T.n_vertices, T.n_cells)
    b = lb.Simulation(p, P, T.n_vertices, T.n_cells)
    a.set_cells(T)
    b.set_cells(T)
    a.advance(n)
    # positions and areas are current after an advance, the lattice fields are not
    got_x = a.fields(lb.LBIB_X | lb.LBIB_AREA)
    assert np.isfinite(got_x["xy"]).all() and (got_x["area"] > 0).all()
    with pytest.raises(lb.LbibError) as e:
        a.fields(lb.LBIB_U)
    assert e.value.code == lb.LBIB_E_STATE
    a.step(1)
    b.step(n + 1)
    fa, fb = a.fields(), b.fields()
    assert max(rel(fa["ux"], fb["ux"]), rel(fa["uy"], fb["uy"])) < tol
    assert rel(fa["rho"] - p.rho0, fb["rho"] - p.rho0) < max(tol, 1e-9)
    assert rel(fa["phi"], fb["phi"]) < tol
    assert np.abs(fa["xy"] - fb["xy"]).max() < tol_x
    # the vertices of the advanced context equal the ones read after the advance,
    # moved by one more step
    assert np.abs(fa["xy"] - got_x["xy"]).max() > 0
    a.close()
    b.close()
