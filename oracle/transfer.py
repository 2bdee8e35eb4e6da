"""Transfer of a state between two grids of the cube by trilinear interpolation (FP64, numpy).

Test infrastructure only (see the package docstring).  The plain definition: along each axis, 1D linear
interpolation (numpy.interp) in physical coordinates between the field's coarse samples extended by its
wall values (Eqs. 4-6), applied axis after axis (trilinear interpolation is the tensor product of the
three 1D interpolations):
  velocity along its own axis: samples on the faces x_f[0..n], zero on both walls;
  velocity across an axis: samples (0, x_c[0..n-1], 1) with zero (no-slip) at the walls;
  T along x: samples (0, x_c, 1) with the Dirichlet values 1 and 0 (Eq. 4);
  T along y and z: the centres only, held constant beyond the first and last (zero flux, Eqs. 5-6).
Then the velocity is projected on the target grid (oracle.projection).  Grid sequencing as in Section 4.1,
which refines its grids and continues solutions from neighbouring states.
"""
from __future__ import annotations

import numpy as np

from . import discretisation as D
from .projection import Projector


def _samples(ax: D.Axis, field: int, axis: int):
    """Coarse sample coordinates along `axis` of `field`, and the left / right wall values (None: none)."""
    if field < 3 and field == axis:
        return ax.xf, 0.0, 0.0          # faces 0..n (walls included in the full array)
    if field < 3:
        return np.concatenate([[0.0], ax.xc, [1.0]]), 0.0, 0.0
    if axis == 0:
        return np.concatenate([[0.0], ax.xc, [1.0]]), 1.0, 0.0
    return ax.xc, None, None


def _targets(ax: D.Axis, field: int, axis: int):
    return ax.xf if (field < 3 and field == axis) else ax.xc


def _interp_axis(a: np.ndarray, np_axis: int, xs, xt, left, right):
    """1D linear interpolation of `a` along numpy axis np_axis from points xs to xt."""
    a = np.moveaxis(a, np_axis, -1)
    if left is not None:
        pad_l = np.full(a.shape[:-1] + (1,), left)
        pad_r = np.full(a.shape[:-1] + (1,), right)
        a = np.concatenate([pad_l, a, pad_r], axis=-1)
    flat = a.reshape(-1, a.shape[-1])
    out = np.stack([np.interp(xt, xs, row) for row in flat])
    return np.moveaxis(out.reshape(a.shape[:-1] + (len(xt),)), -1, np_axis)


def transfer(g_from: D.Grid, q_from, g_to: D.Grid):
    """q_from (full arrays on g_from) -> full arrays on g_to, interpolated and projected."""
    out = []
    for f in range(4):
        a = np.asarray(q_from[f], dtype=np.float64)
        for axis in range(3):
            xs, left, right = _samples(g_from.axes[axis], f, axis)
            if f < 3 and f == axis:
                left = right = None        # the full face array already holds both wall values
            a = _interp_axis(a, 2 - axis, xs, _targets(g_to.axes[axis], f, axis), left, right)
        out.append(a)
    return Projector(g_to).full(out)
