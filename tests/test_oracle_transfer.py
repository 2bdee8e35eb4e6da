"""Pins of the oracle's grid transfer (oracle/transfer.py).

* Conduction (u = 0, T = 1 - x) is linear in x with the wall values of Eq. 4: it transfers exactly.
* A divergence-free velocity from a stream function with no-slip walls, u = s(y) dpsi/dz,
  w = -s(y) dpsi/dx, psi = sin^2(pi x) sin^2(pi z), s(y) = sin^2(pi y), sampled on a coarse grid and transferred to a fixed fine grid, approaches
  the field sampled on the fine grid at second order in the coarse spacing.
* Transferring a divergence-free state onto its own grid returns it.
"""
import numpy as np

import oracle.discretisation as D
from oracle import transfer as TR
from oracle.projection import Projector

PR = 0.71


def test_conduction_transfers_exactly():
    a, b = D.Grid(10, 8, 6, stretch=1.5, Pr=PR), D.Grid(23, 17, 13, stretch=1.5, Pr=PR)
    qb = TR.transfer(a, D.conduction_state(a), b)
    ref = D.conduction_state(b)
    for c in range(4):
        assert np.max(np.abs(qb[c] - ref[c])) <= 1e-14


def _stream_state(g):
    """u = s(y) dpsi/dz, w = -s(y) dpsi/dx with psi = sin^2(pi x) sin^2(pi z), s = sin^2(pi y), exact on
    the staggered points."""
    s2 = lambda t: np.sin(np.pi * t) ** 2
    ds2 = lambda t: np.pi * np.sin(2 * np.pi * t)
    gx, gy, gz = g.axes
    q = [np.zeros(g.full_shape(c)) for c in range(3)] + [np.zeros(g.shape)]
    sy = s2(gy.xc)[None, :, None]      # a y-profile vanishing on the y-walls keeps the field no-slip
    q[0] = s2(gx.xf)[None, None, :] * ds2(gz.xc)[:, None, None] * sy
    q[2] = -ds2(gx.xc)[None, None, :] * s2(gz.xf)[:, None, None] * sy
    q[3] = np.broadcast_to(1.0 - gx.xc[None, None, :], g.shape).copy()
    return q


def test_smooth_field_second_order():
    fine = D.Grid(60, 30, 60, stretch=1.5, Pr=PR)
    ref = _stream_state(fine)
    errs = []
    for n in (10, 20, 40):
        c = D.Grid(n, n // 2, n, stretch=1.5, Pr=PR)
        qf = TR.transfer(c, _stream_state(c), fine)
        errs.append(max(float(np.max(np.abs(qf[k] - ref[k]))) for k in (0, 2)))
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 3.5, errs   # -> 4 (second order)


def test_same_grid_is_the_identity_on_divergence_free_states():
    g = D.Grid(9, 7, 8, stretch=1.5, Pr=PR)
    rng = np.random.default_rng(4)
    q = [rng.standard_normal(g.full_shape(c)) for c in range(3)] + [rng.standard_normal(g.shape)]
    q = D.from_api(g, D.to_api(g, q))
    q = Projector(g).full(q)
    out = TR.transfer(g, q, g)
    for c in range(4):
        assert np.max(np.abs(out[c] - q[c])) <= 1e-12 * max(1.0, float(np.max(np.abs(q[c]))))
