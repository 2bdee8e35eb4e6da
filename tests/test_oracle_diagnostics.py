"""Pins of the oracle's diagnostics on inputs where a wrong implementation gives a different number.

* Symmetry measures (Section 2, Eqs. 7-9): theta = a (y - 1/2) + b (x - 1/2) + c (z - 1/2)^2 on a
  stretched, non-cubic grid.  By hand, with the mirror maps written on the coordinates (not on array
  indices):  theta(x,y,z) - theta(x,1-y,z) = 2a (y - 1/2);  theta(x,y,z) + theta(1-x,y,1-z) =
  2a (y - 1/2) + 2c (z - 1/2)^2;  theta(x,y,z) + theta(1-x,1-y,1-z) = 2c (z - 1/2)^2.  Each maximum is
  taken over the cell centres.  A measure that flips the wrong axes, or that adds where Eq. 7 subtracts,
  gives a different value for at least one of the three.
* Kinetic energy (Eq. 12): each velocity component lives on its own control volumes (the staggered
  face's half-cells on either side along its axis, full cells across).  A unit value on one interior
  face gives 1/2 (x_c[i] - x_c[i-1]) dy_j dz_k, which differs from any cell-width weight on a stretched
  grid; and the energy of u = sin(pi x) sin(pi y) sin(pi z) (likewise v, w) converges to the exact
  integral 1/16 at second order, where a first-order (cell-width) weighting does not.
"""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle import diagnostics as DG

PR = 0.71


def test_symmetry_measures_hand_computed():
    g = D.Grid(9, 12, 7, stretch=1.5, Pr=PR)
    x, y, z = (ax.xc for ax in g.axes)
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    a, b, c = 0.7, -1.3, 2.1
    th = a * (Y - 0.5) + b * (X - 0.5) + c * (Z - 0.5) ** 2 + 0.0 * X * Y * Z
    T = th + (1.0 - X)
    r_ref, r_2d, r_3d = DG.symmetry_measures(g, T)
    f = lambda xx, yy, zz: a * (yy - 0.5) + b * (xx - 0.5) + c * (zz - 0.5) ** 2
    # the maps evaluated on the coordinates themselves
    e_ref = np.max(np.abs(f(X, Y, Z) - f(X, 1.0 - Y, Z)))
    e_2d = np.max(np.abs(f(X, Y, Z) + f(1.0 - X, Y, 1.0 - Z)))
    e_3d = np.max(np.abs(f(X, Y, Z) + f(1.0 - X, 1.0 - Y, 1.0 - Z)))
    # and in closed form from the first centres (the grid is mirrored: 1 - y_c[j] = y_c[n-1-j])
    y0, z0 = g.axes[1].xc[0], g.axes[2].xc[0]
    assert e_ref == pytest.approx(2 * a * (0.5 - y0), rel=1e-13)
    assert e_3d == pytest.approx(2 * c * (0.5 - z0) ** 2, rel=1e-13)
    assert e_2d == pytest.approx(np.max(np.abs(2 * a * (Y - 0.5) + 2 * c * (Z - 0.5) ** 2)), rel=1e-13)
    assert (r_ref, r_2d, r_3d) == pytest.approx((e_ref, e_2d, e_3d), rel=1e-12, abs=1e-14)
    # the three measures are different numbers here, so a permutation of them cannot pass either
    assert min(abs(e_ref - e_2d), abs(e_2d - e_3d), abs(e_ref - e_3d)) > 0.05


@pytest.mark.parametrize("c", [0, 1, 2])
def test_symmetry_measures_single_broken_symmetry(c):
    """A theta that keeps two of the symmetries and breaks exactly one of them (pattern c)."""
    g = D.Grid(8, 10, 6, stretch=1.5, Pr=PR)
    x, y, z = (ax.xc for ax in g.axes)
    X, Y, Z = x[None, None, :] - 0.5, y[None, :, None] - 0.5, z[:, None, None] - 0.5
    # (ref, 2D, 3D) parity of each monomial: x*z keeps ref, flips sign under 2D and 3D -> theta + S theta = 0
    # is required for 2D/3D "kept", theta - S theta = 0 for ref.
    th = [X * Z * Y, X * X * Y, X * Y * Y][c]
    # X Z Y: ref odd (R_ref = 2 max|th|), 2D: + (-X)(Y)(-Z) = +th -> R_2D = 2 max|th|, 3D: (-X)(-Y)(-Z) = -th -> 0
    # X X Y: ref odd, 2D: X^2 Y -> R_2D = 2 max|th|, 3D: X^2 (-Y) = -th -> 0
    # X Y Y: ref even -> 0, 2D: (-X) Y^2 = -th -> 0, 3D: (-X) Y^2 = -th -> 0
    expect = [(2, 2, 0), (2, 2, 0), (0, 0, 0)][c]
    m = float(np.max(np.abs(th)))
    T = th + (1.0 - (X + 0.5))
    got = DG.symmetry_measures(g, T)
    assert got == pytest.approx(tuple(e * m for e in expect), abs=1e-14)


def _unit_face_state(g, comp, idx):
    q = [np.zeros(g.full_shape(c)) for c in range(3)] + [np.zeros(g.shape)]
    q[comp][idx] = 1.0
    return q


@pytest.mark.parametrize("comp,idx", [(0, (2, 3, 1)), (0, (4, 0, 5)), (1, (1, 6, 3)), (2, (5, 2, 7))])
def test_kinetic_energy_of_one_face_value(comp, idx):
    g = D.Grid(9, 8, 7, stretch=1.5, Pr=PR)
    q = _unit_face_state(g, comp, idx)
    k, j, i = idx
    ax = g.axes
    if comp == 0:
        vol = (ax[0].xc[i] - ax[0].xc[i - 1]) * ax[1].dx[j] * ax[2].dx[k]
    elif comp == 1:
        vol = ax[0].dx[i] * (ax[1].xc[j] - ax[1].xc[j - 1]) * ax[2].dx[k]
    else:
        vol = ax[0].dx[i] * ax[1].dx[j] * (ax[2].xc[k] - ax[2].xc[k - 1])
    assert DG.kinetic_energy(g, q) == pytest.approx(0.5 * vol, rel=1e-14)
    # the staggered control volume differs from a cell's on this grid (the pin would catch a dx/dc swap)
    own = [ax[0].dx[i], ax[1].dx[j], ax[2].dx[k]][comp]
    stag = [ax[0].xc[i] - ax[0].xc[i - 1], ax[1].xc[j] - ax[1].xc[j - 1], ax[2].xc[k] - ax[2].xc[k - 1]][comp]
    assert abs(own - stag) > 1e-3 * stag


def _sine_energy(n, comp):
    g = D.Grid(n, n + 2, n + 1, stretch=1.5, Pr=PR)
    s = lambda a: np.sin(np.pi * a)
    q = [np.zeros(g.full_shape(c)) for c in range(3)] + [np.zeros(g.shape)]
    coords = []
    for d in range(3):
        # the component's own axis is sampled on faces, the others at centres
        coords.append(g.axes[d].xf if d == comp else g.axes[d].xc)
    xs, ys, zs = coords
    q[comp] = s(zs)[:, None, None] * s(ys)[None, :, None] * s(xs)[None, None, :]
    return DG.kinetic_energy(g, q)


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_kinetic_energy_converges_at_second_order(comp):
    exact = 0.5 * 0.125          # 1/2 * (1/2)^3
    e1 = abs(_sine_energy(16, comp) - exact)
    e2 = abs(_sine_energy(32, comp) - exact)
    e3 = abs(_sine_energy(64, comp) - exact)
    assert e3 < 2e-3 * exact
    assert e1 / e2 > 3.5 and e2 / e3 > 3.5, (e1, e2, e3)
