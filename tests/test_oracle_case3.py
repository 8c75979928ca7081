"""Oracle pins for species confined by moving membranes (reading c31) and the
concentration-proportional mass source of the paper's validation Case III
(reading c32).

What fixes each result (none of it retypes the oracle's update):
  - a confined species keeps its mass exactly while its cell grows (the
    bounce-back moves nothing across a membrane), nothing appears outside the
    cell, and it does reach the nodes the growing membrane takes in (the
    confinement follows each step's labels, not the first ones);
  - the growth law of Case III: with the source beta C at every node inside
    the cell and the species mass M conserved, dA/dt = beta M, so
    A(T) = A0 + beta M T; the relative area error falls at about first order
    when the lattice is refined in diffusive scaling (diameter x2, T x4,
    beta / 4).
"""
import math

import numpy as np

import lbib_inputs as li

W5 = np.array([1 / 3] + [1 / 6] * 4)


def _case(n, r, T):
    p = li.LatticeParams(nx=n, ny=n, tau=1.0, rho0=1.0, n_species=1)
    p.D[0] = 1.0 / 6.0
    p.noflux, p.noflux_dynamic = 1, 1
    p.mass_beta, p.mass_species = 1.0 / T, 0
    p.pressure_nodes, p.pressure_rho = 1, 1.0
    tis = li.make_tissue([(n / 2, n / 2)], [r], 8 * int(r), 0.0, 0.0, [0])
    X, Y = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
    phi0 = (np.hypot(X - n / 2, Y - n / 2) <= r - 0.1).astype(float)
    pm = np.zeros((n, n), np.uint8)
    pm[0, :] = 1
    pm[:, 0] = 1
    g = np.stack([W5[q] * phi0 for q in range(5)])
    return p, tis, phi0, pm, g


def test_confined_species_follows_the_moving_membrane(orc):
    n, r, T = 64, 8.0, 400
    p, tis, phi0, pm, g = _case(n, r, T)
    lab0, _ = orc.rasterize(n, n, 0, tis.cell_off, tis.xy, tis.src_flag)
    res = orc.run(p, tis, T, g=g, pmask=pm)
    lab1, _ = orc.rasterize(n, n, 0, tis.cell_off, res.xy, tis.src_flag)
    phi = res.phi[0]
    assert abs(phi.sum() / phi0.sum() - 1.0) < 1e-12
    assert np.abs(phi[lab1 == 0]).max() == 0.0
    taken_in = (lab1 > 0) & (lab0 == 0)
    assert taken_in.sum() > 20 and phi[taken_in].min() > 0.0


def _case3_error(orc, n, r, T):
    p, tis, phi0, pm, g = _case(n, r, T)
    A0 = orc.cell_areas(tis.cell_off, tis.xy)[0]
    res = orc.run(p, tis, T, g=g, pmask=pm)
    return res.area[0] / (A0 + p.mass_beta * phi0.sum() * T) - 1.0


def test_case3_linear_growth_converges(orc):
    e1 = _case3_error(orc, 64, 8.0, 400)
    e2 = _case3_error(orc, 128, 16.0, 1600)
    order = math.log2(abs(e1) / abs(e2))
    print(f"relative area error {e1:+.4f} (diameter 16), {e2:+.4f} (32): order {order:.2f}")
    assert abs(e1) < 0.08 and abs(e2) < abs(e1)
    assert 0.6 < order < 1.6
