"""Symmetries (Section 2), symmetry measures (Eqs. 7-9), kinetic energy (Eq. 12), Nusselt number (Eq. 13).

Test infrastructure only (see the package docstring).  All maps act on full
arrays (both walls stored), on which a mirror about 1/2 is a plain flip
because the grid is mirrored exactly.
"""
from __future__ import annotations

import numpy as np

from .discretisation import Grid, interior_velocity

# numpy axes of the full arrays: 0 = z, 1 = y, 2 = x


def _flip(a, axes):
    return np.flip(a, axis=axes).copy() if axes else a.copy()


def sym_ref(q, affine=True):
    """Reflection y -> 1 - y (Section 2 (i)): v changes sign, u, w, T are mirrored."""
    return [_flip(q[0], (1,)), -_flip(q[1], (1,)), _flip(q[2], (1,)), _flip(q[3], (1,))]


def sym_2d(q, affine=True):
    """Rotation by pi about x = z = 1/2 (Section 2 (ii)): (x,y,z) -> (1-x,y,1-z),
    u, w change sign, v is kept and theta = T - (1-x) changes sign, i.e. T -> 1 - T.
    With affine=False the map acts on perturbations (T -> -T)."""
    T = _flip(q[3], (0, 2))
    return [-_flip(q[0], (0, 2)), _flip(q[1], (0, 2)), -_flip(q[2], (0, 2)),
            (1.0 - T) if affine else -T]


def sym_3d(q, affine=True):
    """Centro-symmetry (Section 2 (iii)): (x,y,z) -> (1-x,1-y,1-z), all velocities and theta change sign."""
    T = _flip(q[3], (0, 1, 2))
    return [-_flip(q[0], (0, 1, 2)), -_flip(q[1], (0, 1, 2)), -_flip(q[2], (0, 1, 2)),
            (1.0 - T) if affine else -T]


def theta(grid: Grid, T: np.ndarray) -> np.ndarray:
    """Deviation from conduction theta = T - (1 - x) (Section 2)."""
    return T - (1.0 - grid.axes[0].xc[None, None, :])


def symmetry_measures(grid: Grid, T: np.ndarray):
    """(R_ref, R_2D, R_3D) of Eqs. 7-9 evaluated on cell-centred theta."""
    th = theta(grid, T)
    r_ref = float(np.max(np.abs(th - np.flip(th, axis=1))))
    r_2d = float(np.max(np.abs(th + np.flip(th, axis=(0, 2)))))
    r_3d = float(np.max(np.abs(th + np.flip(th, axis=(0, 1, 2)))))
    return r_ref, r_2d, r_3d


def kinetic_energy(grid: Grid, q) -> float:
    """E_kin = 1/2 int (u^2 + v^2 + w^2) dV (Eq. 12); each component over its own control volumes."""
    gx, gy, gz = grid.axes
    e = 0.0
    vols = [
        gz.dx[:, None, None] * gy.dx[None, :, None] * gx.dc[None, None, :],
        gz.dx[:, None, None] * gy.dc[None, :, None] * gx.dx[None, None, :],
        gz.dc[:, None, None] * gy.dx[None, :, None] * gx.dx[None, None, :],
    ]
    for c in range(3):
        e += float(np.sum(vols[c] * interior_velocity(q, c) ** 2))
    return 0.5 * e


def nusselt_hot(grid: Grid, T: np.ndarray) -> float:
    """Nu = int int [dT/dx]_{x=0} dy dz as printed in Eq. 13 (no sign change), with the
    wall gradient (T_0 - 1) / (dx_0 / 2).  Conduction gives Nu = -1."""
    gx, gy, gz = grid.axes
    g = (T[:, :, 0] - 1.0) / (0.5 * gx.dx[0])
    return float(np.sum(g * gz.dx[:, None] * gy.dx[None, :]))
