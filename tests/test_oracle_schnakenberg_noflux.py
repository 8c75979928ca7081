"""Oracle pins for the Schnakenberg reaction (the Turing-patterning example,
Sec. 4.2) and the half-way bounce-back option for confined species
(noflux_scheme 1; the paper's own no-flux closure of Sec. 6.1 is pinned in
test_oracle_noflux_closure.py).

What fixes each result (none of it retypes the oracle's update):
  - the homogeneous state R* = a + b, L* = b / (a + b)^2 makes both rates
    vanish, so a uniform equilibrium population there is a fixed point;
  - a uniform equilibrium population evolves as phi <- phi + R(phi) (the
    collision of a uniform equilibrium leaves it at equilibrium), so a small
    uniform perturbation of the fixed point follows the linear map I + J with
    J the Jacobian of the rates, derived by hand:
        J = gamma [[-1 + 2 R* L*, R*^2], [-2 R* L*, -R*^2]];
  - a species confined by bounce-back keeps its mass in every domain (no
    population crosses a domain boundary), relaxes to the domain mean
    without reaction, and is unaffected when every node carries the same
    label (under either scheme); a free species moves mass between domains.
"""
import numpy as np
import pytest

import lbib_inputs as li


def _params(nx, ny, gamma=0.05, a=0.1, b=0.9, D=(0.1, 0.3), bc_y=li.BC_PERIODIC, noflux=0,
            reaction=1, scheme=1):
    p = li.LatticeParams(nx=nx, ny=ny, bc_y=bc_y, tau=1.0, rho0=1.0, n_species=2)
    p.noflux_scheme = scheme
    p.D[0], p.D[1] = D
    p.reaction = reaction
    p.schnak = [gamma, a, b]
    p.noflux = noflux
    return p


def _uniform_g(p, phis):
    W5 = np.array([1 / 3] + [1 / 6] * 4)
    g = np.zeros((5 * p.n_species, p.ny, p.nx))
    for s, v in enumerate(phis):
        for q in range(5):
            g[5 * s + q] = W5[q] * v
    return g


def test_schnakenberg_homogeneous_fixed_point(orc):
    a, b = 0.1, 0.9
    p = _params(16, 12, a=a, b=b)
    Rs, Ls = a + b, b / (a + b) ** 2
    g = _uniform_g(p, (Rs, Ls))
    for _ in range(50):
        g, phi = orc.species_step(p, g)
    assert np.abs(phi[0] - Rs).max() < 1e-13
    assert np.abs(phi[1] - Ls).max() < 1e-13


@pytest.mark.parametrize("a,b,gamma", [(0.1, 0.9, 0.05), (0.2, 0.5, 0.02)])
def test_schnakenberg_linearisation(orc, a, b, gamma):
    p = _params(8, 8, gamma=gamma, a=a, b=b)
    Rs, Ls = a + b, b / (a + b) ** 2
    J = gamma * np.array([[-1 + 2 * Rs * Ls, Rs ** 2], [-2 * Rs * Ls, -Rs ** 2]])
    M = np.eye(2) + J
    d0 = np.array([1e-7, -2e-7])
    g = _uniform_g(p, (Rs + d0[0], Ls + d0[1]))
    n = 40
    for _ in range(n):
        g, phi = orc.species_step(p, g)
    # the phi an update returns is the pre-collision moment of that update:
    # after n updates it is the state after n - 1 reaction steps
    got = np.array([phi[0].mean() - Rs, phi[1].mean() - Ls])
    want = np.linalg.matrix_power(M, n - 1) @ d0
    assert np.abs(got - want).max() < 1e-4 * np.abs(want).max()
    # and the field stays uniform
    assert np.ptp(phi[0]) < 1e-15 and np.ptp(phi[1]) < 1e-15


def _domains(nx, ny):
    """Three rectangular domains and the outside (-1)."""
    dom = np.full((ny, nx), -1, np.int32)
    dom[2:9, 3:11] = 0
    dom[10:17, 2:8] = 1
    dom[4:15, 13:21] = 2
    return dom


def _sums(phi, dom):
    return np.array([phi[dom == k].sum() for k in (-1, 0, 1, 2)])


@pytest.mark.parametrize("bc_y", [li.BC_PERIODIC, li.BC_WALLS])
def test_noflux_conserves_domain_mass(orc, bc_y):
    nx, ny = 24, 20
    p = _params(nx, ny, D=(0.2, 0.2), bc_y=bc_y, noflux=1, reaction=0)
    dom = _domains(nx, ny)
    rng = np.random.default_rng(5)
    g = rng.uniform(0.1, 1.0, size=(10, ny, nx))
    phi0 = np.stack([g[0:5].sum(0), g[5:10].sum(0)])
    s0, s1 = _sums(phi0[0], dom), _sums(phi0[1], dom)
    for _ in range(200):
        g, phi = orc.species_step(p, g, dom=dom)
    # confined species: every domain keeps its mass
    assert np.abs(_sums(phi[0], dom) - s0).max() < 1e-11 * s0.max()
    # free species: mass moves between domains, the total is kept
    assert np.abs(_sums(phi[1], dom) - s1).max() > 1e-3 * s1.max()
    assert abs(phi[1].sum() - phi0[1].sum()) < 1e-11 * phi0[1].sum()


def test_noflux_relaxes_to_domain_mean(orc):
    nx, ny = 24, 20
    p = _params(nx, ny, D=(0.3, 0.3), noflux=1, reaction=0)
    dom = _domains(nx, ny)
    rng = np.random.default_rng(6)
    g = rng.uniform(0.0, 1.0, size=(10, ny, nx))
    phi0 = g[0:5].sum(0)
    for _ in range(3000):
        g, phi = orc.species_step(p, g, dom=dom)
    for k in (0, 1, 2):
        m = phi0[dom == k].mean()
        assert np.abs(phi[0][dom == k] - m).max() < 1e-8 * m


@pytest.mark.parametrize("scheme", [0, 1])
def test_noflux_single_domain_is_free(orc, scheme):
    nx, ny = 16, 12
    rng = np.random.default_rng(7)
    g0 = rng.uniform(0.0, 1.0, size=(10, ny, nx))
    dom = np.zeros((ny, nx), np.int32)
    pc = _params(nx, ny, noflux=3, scheme=scheme)
    pf = _params(nx, ny, noflux=0)
    gc, gf = g0.copy(), g0.copy()
    mom = orc.species_moments(pc, gc)
    for _ in range(20):
        mo = np.empty_like(mom)
        gc, phic = orc.species_step(pc, gc, dom=dom, mom=mom, mom_out=mo)
        mom = mo
        gf, phif = orc.species_step(pf, gf)
    assert np.array_equal(phic, phif)


def test_noflux_in_the_coupled_step(orc):
    """Through the fluid step (fluid at rest, no cells): the confined species
    keeps its domain masses as in the species-only update."""
    nx, ny = 24, 20
    p = _params(nx, ny, D=(0.2, 0.2), noflux=1, reaction=0)
    dom = _domains(nx, ny)
    rng = np.random.default_rng(8)
    f, _ = orc.equilibrium_state(p)
    g = rng.uniform(0.1, 1.0, size=(10, ny, nx))
    s0 = _sums(g[0:5].sum(0), dom)
    for _ in range(100):
        f, g, rho, ux, uy, phi = orc.lattice_step(p, f, g, dom=dom)
    assert np.abs(_sums(phi[0], dom) - s0).max() < 1e-11 * s0.max()
