"""Oracle pins for the membrane no-flux condition of confined species as the
paper gives it (Sec. 6.1, no-flux boundary condition for reaction-advection-
diffusion equations; reading c26): a population that would cross a domain
boundary is missing, and it is replaced by the D2Q5 equilibrium of a density
extrapolated to first order from the fluid and a momentum interpolated to
first order between the fluid and zero at the wall point (the half-way point
of the crossing link), both from the previous step's moments.

What fixes each result (none of it retypes the oracle's update):
  - for a density that is linear along the link, first-order extrapolation
    from the two fluid nodes is exact, and the momentum at the node, half a
    link from the wall and three halves from the next fluid node, is one
    third of that node's; a state with no population but the missing one
    shows the missing population itself (the closed form w (phi(x) +
    v.j(x + v)) for a linear phi);
  - D2Q5 is invariant under the lattice's rotations and reflections, so is a
    closure stated without reference to a direction: a rotated (mirrored)
    domain and state give the rotated (mirrored) result;
  - an equilibrium closure leaves a uniform equilibrium in every domain
    unchanged, and a domain without mass or source stays empty;
  - the closure is first order in space: the steady profile of a
    diffusion-decay problem between two membranes converges at first order
    to the closed-form solution with zero-flux (Neumann) conditions at the
    wall points, and with straight membranes the domain mass a transient
    loses falls at first order under refinement.
"""
import numpy as np
import pytest

import lbib_inputs as li

W5 = np.array([1 / 3] + [1 / 6] * 4)


def _params(nx, ny, D=0.1, decay=0.0, bc_y=li.BC_PERIODIC):
    p = li.LatticeParams(nx=nx, ny=ny, bc_y=bc_y, tau=1.0, rho0=1.0, n_species=1)
    p.D[0] = D
    p.decay[0] = decay
    p.noflux = 1
    p.noflux_scheme = 0
    return p


def _steps(orc, p, g, dom, n, src=None, mom=None):
    """n species updates carrying the closure's moments from step to step."""
    if mom is None:
        mom = orc.species_moments(p, g)
    phi = None
    for _ in range(n):
        mo = np.empty_like(mom)
        g, phi = orc.species_step(p, g, src=src, dom=dom, mom=mom, mom_out=mo)
        mom = mo
    return g, phi, mom


@pytest.mark.parametrize("axis", ["x", "y"])
def test_closure_linear_density_closed_form(orc, axis):
    """A strip domain (columns 3..10 of 14), no populations at all, previous
    moments: phi linear, momentum arbitrary along the strip.  The only mass
    after streaming is the closure at the nodes next to a membrane."""
    n = 14
    a, b = 0.7, 0.05
    rng = np.random.default_rng(11)
    J = rng.uniform(-0.2, 0.2, size=n)
    lab = np.zeros(n, np.int32)
    lab[3:11] = 1
    xs = np.arange(n)
    phil = a + b * xs
    if axis == "x":
        p = _params(n, 1)
        dom = lab[None, :]
        mom = np.stack([phil[None, :], J[None, :], np.zeros((1, n))])
    else:
        p = _params(1, n)
        dom = lab[:, None]
        mom = np.stack([phil[:, None], np.zeros((n, 1)), J[:, None]])
    g = np.zeros((5, p.ny, p.nx))
    _, phi = orc.species_step(p, g, dom=dom, mom=mom)
    phi = phi[0].ravel()
    # the closed form at the four nodes next to a membrane: the missing
    # population travels along +e (from the lower side) or -e (from the upper
    # side); the momentum a third of the next node's, projected on that way
    want = np.zeros(n)
    want[3] = W5[1] * (phil[3] + J[4])     # domain 1, entering along +e
    want[10] = W5[1] * (phil[10] - J[9])   # domain 1, entering along -e
    want[2] = W5[1] * (phil[2] - J[1])     # outside, entering along -e
    want[11] = W5[1] * (phil[11] + J[12])  # outside, entering along +e
    assert np.abs(phi - want).max() < 1e-15


def test_closure_thin_domains(orc):
    """Domains one and two nodes wide (the degenerate cases, where fewer
    fluid nodes lie along the link than the extrapolation uses): with one
    fluid node the density is taken from it alone (zeroth order); with none
    (walls on both sides) the momentum is zero and the density is the
    node's own of the previous step."""
    n = 12
    a, b = 0.5, 0.03
    rng = np.random.default_rng(12)
    J = rng.uniform(-0.2, 0.2, size=n)
    lab = np.zeros(n, np.int32)
    lab[3] = 1          # one node wide
    lab[6:8] = 2        # two nodes wide
    phil = a + b * np.arange(n)
    p = _params(n, 1)
    mom = np.stack([phil[None, :], J[None, :], np.zeros((1, n))])
    _, phi = orc.species_step(p, np.zeros((5, 1, n)), dom=lab[None, :], mom=mom)
    phi = phi[0, 0]
    assert abs(phi[3] - 2 * W5[1] * phil[3]) < 1e-15
    assert abs(phi[6] - W5[1] * (phil[7] + J[7])) < 1e-15
    assert abs(phi[7] - W5[1] * (phil[6] - J[6])) < 1e-15


def _blocky_domains(n, seed):
    rng = np.random.default_rng(seed)
    coarse = rng.integers(0, 3, size=(n // 3, n // 3))
    return np.kron(coarse, np.ones((3, 3), np.int64)).astype(np.int32)


def _rot(a):
    """Field rotated by 90 degrees counter-clockwise on a periodic square:
    the value at (x, y) moves to (-y, x)."""
    n = a.shape[-1]
    xs = np.arange(n)
    return a[..., (-xs[None, :]) % n, xs[:, None]]


def test_closure_rotation_and_mirror_invariance(orc):
    n = 12
    p = _params(n, n, D=0.15)
    dom = _blocky_domains(n, 3)
    rng = np.random.default_rng(4)
    g = rng.uniform(0.0, 1.0, size=(5, n, n))
    _, phi, _ = _steps(orc, p, g.copy(), dom, 12)
    # rotation: direction +x -> +y -> -x -> -y -> +x
    perm = {0: 0, 1: 2, 2: 3, 3: 4, 4: 1}
    gr = np.empty_like(g)
    for q in range(5):
        gr[perm[q]] = _rot(g[q])
    _, phir, _ = _steps(orc, p, gr, _rot(dom), 12)
    assert np.abs(phir[0] - _rot(phi[0])).max() < 1e-13
    # mirror x -> -x: +x and -x swap
    mir = lambda a: a[..., (-np.arange(n)) % n]
    gm = np.stack([mir(g[0]), mir(g[3]), mir(g[2]), mir(g[1]), mir(g[4])])
    _, phim, _ = _steps(orc, p, gm, mir(dom), 12)
    assert np.abs(phim[0] - mir(phi[0])).max() < 1e-13


def test_closure_uniform_domains_fixed_point(orc):
    n = 15
    p = _params(n, n, D=0.2)
    dom = _blocky_domains(n, 8)
    level = np.array([0.0, 0.4, 1.3])  # domain 0 holds no mass
    phi0 = level[dom]
    g = np.stack([W5[q] * phi0 for q in range(5)])
    _, phi, _ = _steps(orc, p, g, dom, 25)
    assert np.abs(phi[0] - phi0).max() < 1e-14
    assert np.all(phi[0][dom == 0] == 0.0)


def _strip_steady(orc, L, M=16):
    """Domain of L columns in a periodic lattice of L + M, y-uniform; source
    in the left half of the domain, decay everywhere; diffusive scaling."""
    nx = L + M
    D = 0.1
    k = 40.0 * D / L ** 2
    s = 1.0 / L ** 2
    p = _params(nx, 1, D=D, decay=k)
    p.src_rate[0] = s
    dom = np.zeros((1, nx), np.int32)
    dom[0, :L] = 1
    src = np.zeros((1, nx), np.uint8)
    src[0, : L // 2] = 1
    g = np.zeros((5, 1, nx))
    g, phi, _ = _steps(orc, p, g, dom, int(24 / k), src=src)
    phi = phi[0, 0]
    # closed form: D phi'' - k phi + s [x < xm] = 0 on (-1/2, L - 1/2),
    # phi' = 0 at both wall points
    x = np.arange(L)
    wa, wb, xm = -0.5, L - 0.5, L // 2 - 0.5
    lam = np.sqrt(k / D)
    c1, s1 = np.cosh(lam * (xm - wa)), np.sinh(lam * (xm - wa))
    c2, s2 = np.cosh(lam * (wb - xm)), np.sinh(lam * (wb - xm))
    A = -(s / k) * s2 / (c1 * s2 + s1 * c2)
    B = -A * s1 / s2
    exact = np.where(x < xm, s / k + A * np.cosh(lam * (x - wa)), B * np.cosh(lam * (wb - x)))
    err = np.abs(phi[:L] - exact).max() / np.abs(exact).max()
    # steady mass balance of the domain: production = what leaves it
    prod = (s * (src[0, :L] > 0) - k * phi[:L]).sum()
    return err, prod / (s * (L // 2)), phi[L:]


def test_closure_first_order_neumann_profile(orc):
    errs = []
    for L in (16, 32, 64):
        err, leak, outside = _strip_steady(orc, L)
        errs.append(err)
        assert abs(leak) < 1e-9          # no net flux through the membranes
        assert np.all(outside == 0.0)    # nothing reaches the other domain
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 0.6) and np.all(orders < 1.4), (errs, orders)
    assert errs[-1] < 1e-2


def test_closure_transient_leak_first_order(orc):
    """Pure diffusion in a square domain (straight membranes) from a profile
    with zero normal gradient at the wall points: the exact solution keeps
    its mass; the domain mass lost over the same diffusive time falls at
    about first order."""
    leaks = []
    for R in (6, 12, 24):
        n = 2 * R + 8
        p = _params(n, n, D=0.1)
        yy, xx = np.mgrid[0:n, 0:n]
        c = (n - 1) / 2
        inside = (np.abs(xx - c) < R) & (np.abs(yy - c) < R)
        dom = inside.astype(np.int32)
        # the wall points sit at c +- R on both axes
        phi0 = np.where(inside, 1.0 + np.cos(np.pi * (xx - c) / R) * np.cos(np.pi * (yy - c) / R),
                        0.0)
        g = np.stack([W5[q] * phi0 for q in range(5)])
        M0 = phi0.sum()
        _, phi, _ = _steps(orc, p, g, dom, int(0.5 * R * R / 0.1))
        leaks.append(abs(phi[0][inside].sum() - M0) / M0)
    leaks = np.array(leaks)
    assert np.all(np.diff(leaks) < 0), leaks
    assert np.log2(leaks[0] / leaks[-1]) / 2 > 0.7, leaks
    assert leaks[-1] < 0.02
