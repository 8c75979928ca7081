"""FP16 storage: the two- and four-nodes-per-thread lattice updates against
the one-node-per-thread update (lbib_set_lattice_variant 2 and 4 vs 1).

All evaluate the same collision (Sec. 6.1, Eq. bgkequation) with the same
FP32 operations per node; the pair and quad updates only change how the
stored halves move (32- or 64-bit words, shifted words assembled from
neighbouring lanes).  So on
the same state, without cells (no atomic spreading, whose summation order
varies from run to run), every stored population and every output field must
be bit-identical.  The states are random stored values (not a rest state) so
that every direction carries a different value at every node; widths are
chosen so that warps end inside a row, a row holds a single partial warp,
and the last pair or quad of a row wraps to x = 0 (widths that are not a
multiple of four run the pair update under variant 4).  With cells, where the
spread force is summed by atomics in varying order, the variants agree to far
below the FP16 error bound; a width of 192 (rows starting at odd multiples of
64 nodes) makes a quad warp's groups straddle two mask words.
"""
import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu

ALL_LATTICE = 1 | 2 | 4


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import build, lbib
    build.build()
    lbib.load()
    return lbib


def _params(nx, ny, walls, S, forcing, body):
    p = li.LatticeParams(nx=nx, ny=ny, bc_y=li.BC_WALLS if walls else li.BC_PERIODIC,
                         tau=0.7, rho0=1.0, n_species=S)
    for s in range(S):
        p.D[s] = 0.05 + 0.03 * s
        p.decay[s] = 1e-3
        for b in range(S):
            if b != s:
                p.react[s][b] = 0.01 * (s - b)
    p.forcing = forcing
    p.body_force = body
    return p


def _random_state(lb, p, seed):
    """A state blob of the FP16 context with random stored populations."""
    sim = lb.Simulation(p, lb.LBIB_FP16, 0, 0)
    blob = sim.get_state().copy()
    sim.close()
    pitch = (p.nx + 63) // 64 * 64
    plane = pitch * p.ny + 1536 // 2
    n = (9 + 5 * p.n_species) * plane
    rng = np.random.Generator(np.random.PCG64(seed))
    vals = rng.uniform(-0.5, 0.5, size=n).astype(np.float16)
    blob[16:16 + 2 * n] = vals.view(np.uint8)
    return blob


def _run(lb, p, blob, variant, n):
    sim = lb.Simulation(p, lb.LBIB_FP16, 0, 0)
    sim.set_state(blob)
    sim.set_lattice_variant(variant)
    sim.step(n)
    out = sim.fields(ALL_LATTICE)
    st = sim.get_state()
    sim.close()
    return out, st


@pytest.mark.parametrize("nx,ny,walls,S,forcing,body", [
    (200, 40, True, 2, 0, (1e-5, 0.0)),      # 100 pairs: the 4th warp holds 4 lanes
    (512, 24, False, 1, 0, (0.0, 0.0)),      # whole warps, periodic wrap at both ends
    (130, 33, True, 3, 1, (2e-6, -1e-6)),    # 65 pairs: a warp of one lane; paper forcing
    (66, 20, False, 4, 0, (0.0, 3e-6)),      # 33 pairs, four species
    (1000, 16, False, 0, 1, (1e-5, 1e-5)),   # four CTAs per row, the last one partial
    (136, 30, True, 2, 0, (1e-5, 2e-6)),     # 34 quads: a warp and a two-lane warp
    (8, 12, False, 1, 1, (1e-6, 0.0)),       # two quads per row: every edge wraps or meets
    (192, 18, False, 1, 0, (3e-6, 0.0)),     # rows at odd multiples of 64 nodes
])
@pytest.mark.parametrize("variant", [2, 4])
def test_pairs_bitwise_without_cells(lb, nx, ny, walls, S, forcing, body, variant):
    p = _params(nx, ny, walls, S, forcing, body)
    blob = _random_state(lb, p, seed=nx * 7 + S)
    for n in (1, 6):   # a single launch, then graph chunks and the tail
        a, sa = _run(lb, p, blob, variant, n)
        b, sb = _run(lb, p, blob, 1, n)
        assert np.array_equal(sa, sb), f"stored state differs after {n} steps"
        for k in ("rho", "ux", "uy") + (("phi",) if S else ()):
            assert np.array_equal(a[k], b[k]), f"{k} differs after {n} steps"
        assert np.isfinite(a["ux"]).all()


def _rel(a, b):
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / s) if s > 0 else float(np.abs(a - b).max())


@pytest.mark.parametrize("wl", ["walls_2species", "periodic_1species", "walls_192"])
@pytest.mark.parametrize("variant", [2, 4])
def test_pairs_with_cells_match_single(lb, wl, variant):
    if wl == "walls_2species":
        w = li.config2(nx=200, ny=150, n_cells_side=4)
    elif wl == "walls_192":
        w = li.config2(nx=192, ny=160, n_cells_side=4)
    else:
        w = li.config3(n=512)
    p, T = w.params, w.tissue
    res = {}
    for variant in (variant, 1):
        sim = lb.Simulation(p, lb.LBIB_FP16, T.n_vertices, T.n_cells)
        sim.set_cells(T)
        sim.set_lattice_variant(variant)
        sim.step(1)
        first = sim.fields(32)
        sim.step(19)
        res[variant] = (first, sim.fields(1 | 2 | 4 | 8 | 32 | 64))
        sim.close()
    (f2, a), (f1, b) = res[variant], res[1]
    assert np.array_equal(f2["id"], f1["id"])      # same X^0: identical labels
    assert _rel(a["ux"], b["ux"]) < 1e-3 and _rel(a["uy"], b["uy"]) < 1e-3
    assert _rel(a["phi"], b["phi"]) < 1e-3
    assert np.abs(a["xy"] - b["xy"]).max() < 1e-6


def test_variant_rejects_other_values(lb):
    w = li.config1()
    sim = lb.Simulation(w.params, lb.LBIB_FP16, 0, 0)
    for bad in (3, -1, 8):
        with pytest.raises(lb.LbibError):
            sim.set_lattice_variant(bad)
    sim.close()
