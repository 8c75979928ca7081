"""Species confined by the moving membranes (reading c31) and the
concentration-proportional mass source (reading c32): GPU parity against the
FP64 oracle, and the paper's validation Case III (Sec. 6.3).

  - a growing cell holding one species, confined by each step's labels, with
    the source beta C inside: FP64 within 1e-10 (velocity, density,
    concentration, positions, areas, labels) after 120 steps, in one call and
    split over calls of both buffer parities; FP32 within the FP32 bounds
    (u, phi 1e-4), FP16 shifted storage within its bounds (u 3e-2, phi
    1e-2), the positions of both within the relative velocity bound times
    the largest displacement (the cell grows: vertices move by about one
    lattice unit; FP32 measured 1.8e-6);
  - on the GPU the species mass stays constant (FP64: 1e-12) and nothing
    appears outside the cell;
  - contexts with moving confinement refuse a static domain plane;
  - Case III: with the species mass M conserved, dA/dt = beta M, so
    A(T) = A0 + beta M T; four refinements (diameter 10 -> 80, T x4, beta / 4),
    FP32: the area reaches the expected value within 8% at every level and
    the relative error falls at an observed order within [0.7, 1.4]; the
    coarsest level matches the FP64 oracle within 1e-4.
"""
import math

import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu

ALL = 1 | 2 | 4 | 8 | 16 | 32 | 64 | 128
W5 = np.array([1 / 3] + [1 / 6] * 4)


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


def _small():
    n, r = 64, 8.0
    p = li.LatticeParams(nx=n, ny=n, tau=1.0, rho0=1.0, n_species=1)
    p.D[0] = 1.0 / 6.0
    p.noflux, p.noflux_dynamic = 1, 1
    p.mass_beta, p.mass_species = 1.0 / 400, 0
    p.pressure_nodes, p.pressure_rho = 1, 1.0
    T = li.make_tissue([(n / 2 + 0.3, n / 2 - 0.2)], [r], 64, 0.0, 0.0, [0])
    X, Y = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
    phi0 = (np.hypot(X - n / 2 - 0.3, Y - n / 2 + 0.2) <= r - 0.1).astype(float)
    pm = np.zeros((n, n), np.uint8)
    pm[0, :] = 1
    pm[:, 0] = 1
    return p, T, phi0, pm


def _gpu(lb, p, T, phi0, pm, prec, calls):
    sim = lb.Simulation(p, prec, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.set_species(0, phi0)
    sim.set_pressure_nodes(pm)
    for n in calls:
        sim.step(n)
    out = sim.fields(ALL)
    sim.close()
    return out


def _oracle(orc, p, T, phi0, pm, n):
    g = np.stack([W5[q] * phi0 for q in range(5)])
    return orc.run(p, T, n, g=g, pmask=pm)


@pytest.mark.parametrize("calls", [(120,), (57, 63), (1, 60, 59)])
def test_moving_confinement_fp64(lb, orc, calls):
    p, T, phi0, pm = _small()
    ref = _oracle(orc, p, T, phi0, pm, 120)
    got = _gpu(lb, p, T, phi0, pm, lb.LBIB_FP64, calls)
    assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < 1e-10
    assert rel(got["rho"], ref.rho) < 1e-12
    assert rel(got["phi"], ref.phi) < 1e-10
    assert np.abs(got["xy"] - ref.xy).max() < 1e-10
    assert rel(got["area"], ref.area) < 1e-12
    assert np.array_equal(got["id"], ref.id)
    # the species stays in its cell and keeps its mass
    phi = got["phi"][0]
    assert abs(phi.sum() / phi0.sum() - 1.0) < 1e-12
    assert np.abs(phi[got["id"] == 0]).max() == 0.0
    assert ref.area[0] > 1.05 * orc.cell_areas(T.cell_off, T.xy)[0]


@pytest.mark.parametrize("prec,tu,tp", [("fp32", 1e-4, 1e-4), ("fp16", 3e-2, 1e-2)])
def test_moving_confinement_reduced(lb, orc, prec, tu, tp):
    p, T, phi0, pm = _small()
    ref = _oracle(orc, p, T, phi0, pm, 120)
    tx = tu * np.abs(ref.xy - T.xy).max()
    got = _gpu(lb, p, T, phi0, pm, lb.PRECISIONS[prec], (120,))
    eu = max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy))
    ep = rel(got["phi"], ref.phi)
    ex = np.abs(got["xy"] - ref.xy).max()
    print(f"{prec}: u {eu:.2e}  phi {ep:.2e}  X {ex:.2e}")
    assert eu < tu and ep < tp and ex < tx


def test_moving_confinement_refuses_static_domains(lb):
    p, T, phi0, pm = _small()
    sim = lb.Simulation(p, lb.LBIB_FP32, T.n_vertices, T.n_cells)
    with pytest.raises(lb.LbibError):
        sim.set_domains(np.zeros((p.ny, p.nx), np.int32))
    sim.close()


def _case3_ratio(lb, w):
    T = w.tissue
    sim = lb.Simulation(w.params, lb.LBIB_FP32, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    sim.set_species(0, w.phi0[0])
    sim.set_pressure_nodes(w.pressure_mask)
    a0 = sim.fields(lb.LBIB_AREA)["area"][0]
    sim.step(w.n_steps)
    a1 = sim.fields(lb.LBIB_AREA)["area"][0]
    sim.close()
    expect = (a0 + w.params.mass_beta * w.phi0.sum() * w.n_steps) / a0
    return a1 / a0, expect


def test_case3_growth_converges(lb):
    errs = []
    for k in range(4):
        r, expect = _case3_ratio(lb, li.case3(k))
        e = r / expect - 1.0
        print(f"level {k}: area ratio {r:.5f} (expected {expect:.5f}), relative error {e:+.5f}")
        assert abs(e) < 0.08
        errs.append(abs(e))
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(3)]
    print("orders", ["%.2f" % o for o in orders])
    for o in orders:
        assert 0.7 < o < 1.4


def test_case3_coarsest_matches_oracle(lb, orc):
    w = li.case3(0)
    r_gpu, _ = _case3_ratio(lb, w)
    T = w.tissue
    a0 = orc.cell_areas(T.cell_off, T.xy)[0]
    g = np.stack([W5[q] * w.phi0[0] for q in range(5)])
    ref = orc.run(w.params, T, w.n_steps, g=g, pmask=w.pressure_mask)
    r_orc = ref.area[0] / a0
    print(f"GPU {r_gpu:.6f}  oracle {r_orc:.6f}")
    assert abs(r_gpu / r_orc - 1.0) < 1e-4
