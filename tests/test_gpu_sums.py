"""FP64 conservation sums on the GPU (lbib_get_sums) against the oracle and
against what the method fixes.

  - one-cell tissue (config 1, FP64, periodic): global sum rho, sum rho u,
    sum phi and the per-cell sums of rho and phi agree with the same sums of
    the FP64 oracle's fields within 1e-12 relative (rho u: 1e-12 of
    sum |rho u|, it sums to nearly zero);
  - periodic lattice, FP64: the total mass is conserved (1e-13 relative
    between two calls), and under a uniform body force F the total momentum
    of step n is (n - 1/2) N F (Guo forcing: the populations gain N F per
    step, the velocity of the step carries half the step's force);
  - the 1024^2 walled tissue in FP32: the kernel's sums equal the same sums
    over the fields lbib_get_fields returns (1e-12 relative: only the
    summation order differs), and the per-cell sums add up to the sum over
    the labelled nodes;
  - a non-finite concentration is counted, not hidden.
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


def test_sums_match_oracle_fp64(lb, orc):
    w = li.config1()
    p, T = w.params, w.tissue
    n = 200
    ref = orc.run(p, T, n)
    rg, rc = orc.sums(p, ref, T.n_cells)
    sim = lb.Simulation(p, lb.LBIB_FP64, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.step(n)
    g, c, bad = sim.sums()
    sim.close()
    assert bad == 0
    assert abs(g[0] - rg[0]) < 1e-12 * abs(rg[0])
    scale_j = np.abs(ref.rho * ref.ux).sum() + np.abs(ref.rho * ref.uy).sum()
    assert np.abs(g[1:3] - rg[1:3]).max() < 1e-12 * scale_j
    assert abs(g[3] - rg[3]) < 1e-12 * abs(rg[3])
    assert np.abs(c - rc).max() < 1e-12 * np.abs(rc).max()
    assert rc[0, 1] > 0  # the source cell holds species mass


def test_mass_conserved_and_momentum_from_body_force(lb):
    w = li.config1()
    p, T = w.params, w.tissue
    F = (2.0e-6, -1.0e-6)
    p.body_force = F
    N = p.nx * p.ny
    sim = lb.Simulation(p, lb.LBIB_FP64, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.step(30)
    g1, _, _ = sim.sums()
    sim.step(45)
    g2, _, _ = sim.sums()
    sim.close()
    assert abs(g2[0] - g1[0]) < 1e-13 * g1[0]
    assert abs(g1[0] - N * p.rho0) < 1e-12 * N
    # the cells' forces sum to zero: the momentum is the body force's
    for n, g in ((30, g1), (75, g2)):
        want = (n - 0.5) * N * np.array(F)
        assert np.abs(g[1:3] - want).max() < 1e-10 * np.abs(want).max(), (n, g[1:3], want)


def test_sums_of_returned_fields_fp32(lb):
    w = li.config2()
    p, T = w.params, w.tissue
    sim = lb.Simulation(p, lb.LBIB_FP32, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.step(7)
    g, c, bad = sim.sums()
    f = sim.fields(lb.LBIB_RHO | lb.LBIB_U | lb.LBIB_PHI | lb.LBIB_ID)
    sim.close()
    assert bad == 0
    S = p.n_species
    want = np.array([f["rho"].sum(), (f["rho"] * f["ux"]).sum(), (f["rho"] * f["uy"]).sum()] +
                    [f["phi"][s].sum() for s in range(S)])
    assert abs(g[0] - want[0]) < 1e-12 * want[0]
    for s in range(S):
        assert abs(g[3 + s] - want[3 + s]) < 1e-12 * np.abs(f["phi"][s]).sum()
    scale_j = np.abs(f["rho"] * f["ux"]).sum() + np.abs(f["rho"] * f["uy"]).sum()
    assert np.abs(g[1:3] - want[1:3]).max() < 1e-12 * scale_j
    inside = f["id"] > 0
    assert abs(c[:, 0].sum() - f["rho"][inside].sum()) < 1e-12 * f["rho"][inside].sum()
    for cc in (0, 17, T.n_cells - 1):
        m = f["id"] == cc + 1
        assert abs(c[cc, 0] - f["rho"][m].sum()) < 1e-12 * f["rho"][m].sum()
        for s in range(S):
            assert abs(c[cc, 1 + s] - f["phi"][s][m].sum()) <= 1e-12 * max(
                np.abs(f["phi"][s][m]).sum(), 1e-300)


def test_nonfinite_counted(lb):
    w = li.config1()
    p, T = w.params, w.tissue
    sim = lb.Simulation(p, lb.LBIB_FP64, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    phi0 = np.zeros((p.ny, p.nx))
    phi0[5, 7] = np.nan
    sim.set_species(0, phi0)
    sim.step(1)
    g, _, bad = sim.sums()
    sim.close()
    assert bad >= 1
    assert np.isnan(g[3])


def test_sums_need_an_output_step(lb):
    w = li.config1()
    sim = lb.Simulation(w.params, lb.LBIB_FP64, w.tissue.n_vertices, w.tissue.n_cells)
    sim.set_cells(w.tissue)
    sim.advance(3)
    with pytest.raises(lb.LbibError) as e:
        sim.sums()
    assert e.value.code == lb.LBIB_E_STATE
    sim.step(1)
    g, _, _ = sim.sums()
    assert g[0] > 0
    sim.close()
