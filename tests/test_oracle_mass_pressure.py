"""Oracle pins for mass sources, the cell area controller (Sec. 3.2.3) and
internal pressure nodes (Sec. 6.1; readings c29 and c30).

What fixes each result (none of it retypes the oracle's update):
  - at rest, a mass source S at one node leaves the node with w_q (rho0 + S)
    in every direction and changes no other node: the weights of the
    equilibrium, and the equilibrium is a fixed point of the collision;
  - with random populations the lattice gains exactly the summed source and
    no momentum (mass and momentum balance of the stream + collide update);
  - a pressure node holds the prescribed density and keeps the velocity of
    the populations that streamed into it (gamma cancels in u); streaming is
    done here independently with np.roll, and every other node keeps the
    density of what streamed into it;
  - the paper's validation Case II: a uniform source S inside a circular
    cell grows its area as A0 exp(S t) when the excess mass can leave
    through pressure nodes (here a frame at the periodic seam);
  - the proportional controller S = alpha (A0 - A) brings the cell to its
    set-point area from below and from above (its fixed point);
  - the paper's validation Case I: a point source q at the cell centre grows
    the area linearly, A(t) = A0 + q t, with a relative error that falls with
    refinement.
"""
import math

import numpy as np
import pytest

import lbib_inputs as li

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _rest(p):
    return np.repeat(W9 * p.rho0, p.nx * p.ny).reshape(9, p.ny, p.nx).copy()


def test_source_at_rest_adds_the_weights(orc):
    p = li.LatticeParams(nx=16, ny=12, tau=0.8, rho0=1.0)
    f = _rest(p)
    ms = np.zeros((p.ny, p.nx))
    ms[5, 7] = 0.01
    fo, _, rho, ux, uy, _ = orc.lattice_step(p, f, np.zeros(1), msrc=ms)
    assert np.abs(fo[:, 5, 7] - W9 * 1.01).max() < 1e-15
    other = np.ones((p.ny, p.nx), bool)
    other[5, 7] = False
    assert np.abs(fo[:, other] - W9[:, None]).max() < 1e-15
    # the moments of this step are those before the source
    assert np.abs(rho - 1.0).max() < 1e-15 and np.abs(ux).max() < 1e-15


def test_source_mass_and_momentum_balance(orc):
    p = li.LatticeParams(nx=20, ny=18, tau=0.7, rho0=1.0)
    rng = np.random.default_rng(5)
    f = _rest(p) * (1.0 + 0.1 * rng.uniform(-1, 1, size=(9, p.ny, p.nx)))
    ms = 1e-3 * rng.uniform(-1, 1, size=(p.ny, p.nx))
    fo, *_ = orc.lattice_step(p, f, np.zeros(1), msrc=ms)
    assert abs(fo.sum() - (f.sum() + ms.sum())) < 1e-12 * f.sum()
    for c in (CX, CY):
        mom_in = (f * c[:, None, None]).sum()
        mom_out = (fo * c[:, None, None]).sum()
        assert abs(mom_out - mom_in) < 1e-13


def test_pressure_node_density_and_velocity(orc):
    p = li.LatticeParams(nx=20, ny=16, tau=0.9, rho0=1.0)
    p.pressure_rho = 1.05
    rng = np.random.default_rng(6)
    f = _rest(p) * (1.0 + 0.2 * rng.uniform(-1, 1, size=(9, p.ny, p.nx)))
    pm = np.zeros((p.ny, p.nx), np.uint8)
    pm[3, 4] = pm[10, 17] = pm[0, 0] = 1
    _, _, rho, ux, uy, _ = orc.lattice_step(p, f, np.zeros(1), pmask=pm)
    # streaming by pulling, done independently: f_q(x) <- f_q(x - c_q)
    pulled = np.stack([np.roll(f[q], (CY[q], CX[q]), axis=(0, 1)) for q in range(9)])
    rp = pulled.sum(axis=0)
    uxp = (pulled * CX[:, None, None]).sum(axis=0) / rp
    uyp = (pulled * CY[:, None, None]).sum(axis=0) / rp
    on = pm.astype(bool)
    assert np.abs(rho[on] - 1.05).max() < 1e-14
    assert np.abs(rho[~on] - rp[~on]).max() < 1e-14
    assert np.abs(ux - uxp).max() < 1e-14 and np.abs(uy - uyp).max() < 1e-14


def _one_cell(n, r, n_vert=64):
    T = li.make_tissue([(n / 2 + 0.3, n / 2 - 0.2)], [r], n_vert, 0.0, 0.0, [0])
    return T


def _frame(n):
    pm = np.zeros((n, n), np.uint8)
    pm[0, :] = 1
    pm[:, 0] = 1
    return pm


def _case2_error(orc, n, r, S, T):
    p = li.LatticeParams(nx=n, ny=n, tau=1.0, rho0=1.0)
    p.pressure_nodes, p.pressure_rho = 1, 1.0
    p.mass_sources = 1
    tis = _one_cell(n, r, 8 * int(r))
    A0 = orc.cell_areas(tis.cell_off, tis.xy)[0]
    res = orc.run(p, tis, T, mass_rate=np.array([S]), pmask=_frame(n))
    return res.area[0] / A0 / math.exp(S * T) - 1.0


def test_uniform_source_grows_exponentially(orc):
    """Validation Case II: dA/dt = S A, so A(t) = A0 exp(S t); the relative
    area error falls at about first order (the paper: about 1) when the
    lattice is refined in diffusive scaling (diameter x2, S / 4, T x 4)."""
    e1 = _case2_error(orc, 64, 8.0, 1e-3, 400)
    e2 = _case2_error(orc, 128, 16.0, 2.5e-4, 1600)
    order = math.log2(abs(e1) / abs(e2))
    print(f"relative area error {e1:+.4f} (diameter 16), {e2:+.4f} (32): order {order:.2f}")
    assert abs(e1) < 0.06 and abs(e2) < abs(e1)
    assert 0.7 < order < 1.3
    # without the source nothing grows
    n = 64
    p = li.LatticeParams(nx=n, ny=n, tau=1.0, rho0=1.0)
    p.pressure_nodes, p.pressure_rho, p.mass_sources = 1, 1.0, 1
    tis = _one_cell(n, 8.0)
    A0 = orc.cell_areas(tis.cell_off, tis.xy)[0]
    r0 = orc.run(p, tis, 400, mass_rate=np.array([0.0]), pmask=_frame(n))
    assert abs(r0.area[0] / A0 - 1.0) < 1e-3


@pytest.mark.parametrize("target_ratio", [1.3, 0.75])
def test_area_controller_reaches_its_set_point(orc, target_ratio):
    n = 64
    p = li.LatticeParams(nx=n, ny=n, tau=1.0, rho0=1.0)
    p.pressure_nodes, p.pressure_rho = 1, 1.0
    p.mass_sources, p.mass_alpha = 1, 1e-4
    tis = _one_cell(n, 8.0)
    A0 = orc.cell_areas(tis.cell_off, tis.xy)[0]
    At = target_ratio * A0
    r = orc.run(p, tis, 800, mass_rate=np.array([0.0]), target_area=np.array([At]),
                pmask=_frame(n))
    print(f"target {At:.2f}, reached {r.area[0]:.2f} from {A0:.2f}")
    assert abs(r.area[0] / At - 1.0) < 0.01


def _case1_error(orc, n, r, q, T):
    p = li.LatticeParams(nx=n, ny=n, tau=1.0, rho0=1.0)
    p.pressure_nodes, p.pressure_rho = 1, 1.0
    tis = li.make_tissue([(n / 2, n / 2)], [r], 8 * int(r), 0.0, 0.0, [0])
    A0 = orc.cell_areas(tis.cell_off, tis.xy)[0]
    ns = np.zeros((n, n))
    ns[n // 2, n // 2] = q
    res = orc.run(p, tis, T, pmask=_frame(n), node_source=ns)
    return res.area[0] / (A0 + q * T) - 1.0


def test_point_source_grows_linearly(orc):
    """Validation Case I: dA/dt = q for a point source of strength q, so
    A(t) = A0 + q t; refining in diffusive scaling (diameter x2, T x4, q per
    step fixed) the relative area error falls."""
    e1 = _case1_error(orc, 64, 8.0, 0.05, 300)
    e2 = _case1_error(orc, 128, 16.0, 0.05, 1200)
    order = math.log2(abs(e1) / abs(e2))
    print(f"relative area error {e1:+.4f} (diameter 16), {e2:+.4f} (32): order {order:.2f}")
    assert abs(e1) < 0.005 and abs(e2) < abs(e1)
    assert 0.8 < order < 2.2
