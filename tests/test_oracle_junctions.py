"""Oracle pins for the cell junctions of Eq. celljunctionforce (Sec. 3.2.4;
renewal and partner rule: reading c28).

Two rectangles-as-polygons facing each other across a gap g, with vertices
placed so that the closest vertex of the other cell is known by
construction:
  - every vertex of a facing edge pairs with its mirror vertex, and the
    junction force on it is k (g - l0) along the gap (closed form);
  - nothing pairs when g >= l_max, and vertices farther than l_max from the
    other cell have no partner;
  - the periodic image in x counts (a pair across the seam);
  - mutual pairs carry equal and opposite forces;
  - in the coupled step the junctions add exactly these forces to the
    polygon forces at the renewal step.
"""
import numpy as np

import lbib_inputs as li


def _two_boxes(gap, x0=10.0, y0=10.0, w=6.0, h=4.0, n_side=4):
    """Two CCW rectangles [x0, x0+w] x [y0, y0+h] and the one to its right
    starting at x0 + w + gap, each with n_side vertices per edge."""
    def box(xa):
        pts = []
        for k in range(n_side):                       # bottom, left to right
            pts.append((xa + w * k / n_side, y0))
        for k in range(n_side):                       # right, bottom to top
            pts.append((xa + w, y0 + h * k / n_side))
        for k in range(n_side):                       # top, right to left
            pts.append((xa + w - w * k / n_side, y0 + h))
        for k in range(n_side):                       # left, top to bottom
            pts.append((xa, y0 + h - h * k / n_side))
        return np.array(pts)
    a, b = box(x0), box(x0 + w + gap)
    xy = np.concatenate([a, b])
    off = np.array([0, len(a), len(a) + len(b)], np.int32)
    return off, xy


def test_facing_edges_pair_with_their_mirror(orc):
    g, n = 1.5, 4
    off, xy = _two_boxes(g, n_side=n)
    part = orc.junction_partners(64, 48, 0, off, xy, lmax=2.0)
    nA = off[1]
    # right edge of A: local indices n .. 2n-1 (y0 + h k/n), plus the corner
    # at index 2n (top right); left edge of B runs top to bottom from 3n
    for k in range(n):
        i = n + k
        y = xy[i, 1]
        js = [j for j in range(nA, len(xy)) if abs(xy[j, 0] - (xy[i, 0] + g)) < 1e-12
              and abs(xy[j, 1] - y) < 1e-12]
        assert len(js) == 1 and part[i] == js[0]
    # vertices farther than l_max from B (left edge of A) have none
    for i in range(3 * n, 4 * n):
        assert part[i] == -1


def test_force_closed_form_and_cutoff(orc):
    g, n, k, l0 = 1.5, 4, 0.3, 0.5
    off, xy = _two_boxes(g, n_side=n)
    part = orc.junction_partners(64, 48, 0, off, xy, lmax=2.0)
    F = orc.junction_forces(64, 48, 0, xy, part, k, l0, 2.0)
    for kk in range(1, n):           # right edge of A (interior vertices)
        i = n + kk
        assert abs(F[i, 0] - k * (g - l0)) < 1e-14 and abs(F[i, 1]) < 1e-14
    # at g >= l_max nothing pairs
    off2, xy2 = _two_boxes(2.5, n_side=n)
    part2 = orc.junction_partners(64, 48, 0, off2, xy2, lmax=2.0)
    assert (part2 == -1).all()
    assert np.abs(orc.junction_forces(64, 48, 0, xy2, part2, k, l0, 2.0)).max() == 0.0


def test_mutual_pairs_equal_and_opposite(orc):
    off, xy = _two_boxes(1.2, n_side=5)
    part = orc.junction_partners(64, 48, 0, off, xy, lmax=2.0)
    F = orc.junction_forces(64, 48, 0, xy, part, 0.2, 0.4, 2.0)
    mutual = [(i, j) for i, j in enumerate(part) if j >= 0 and part[j] == i and i < j]
    assert len(mutual) >= 4
    for i, j in mutual:
        assert np.abs(F[i] + F[j]).max() < 1e-15


def test_periodic_image_in_x(orc):
    nx = 32
    off, xy = _two_boxes(1.0, x0=25.0, w=6.0)     # B starts at 32 = the seam
    xy[off[1]:, 0] -= nx                         # B drawn at x in [0, 6)
    part = orc.junction_partners(nx, 48, 0, off, xy, lmax=2.0)
    assert (part[4:8] >= off[1]).all()           # A's right edge finds B across the seam
    F = orc.junction_forces(nx, 48, 0, xy, part, 0.3, 0.5, 2.0)
    assert F[5, 0] > 0                           # pulled towards +x, across the seam


def test_coupled_step_adds_the_junction_forces(orc):
    off, xy = _two_boxes(1.5, x0=20.0, y0=20.0, n_side=4)
    T = li.Tissue(off, xy.copy(), li.edge_lengths(off, xy), np.full(xy.shape[0], 0.01),
                  np.zeros(2), np.zeros(2, np.uint8))
    p = li.LatticeParams(nx=64, ny=48, tau=1.0)
    p.junction_k, p.junction_l0, p.junction_lmax, p.junction_period = 0.3, 0.5, 2.0, 5
    r = orc.run(p, T, 1)
    Fpoly = orc.polygon_forces(off, xy, T.rest_len, T.k_spring, T.pressure)
    part = orc.junction_partners(64, 48, 0, off, xy, 2.0)
    Fj = orc.junction_forces(64, 48, 0, xy, part, 0.3, 0.5, 2.0)
    assert np.abs(r.Fv - (Fpoly + Fj)).max() < 1e-15
    assert np.abs(Fj).max() > 0
