"""Grid, residual F, Jacobian-vector product J.v, divergence D and gradient G (FP64, numpy).

Test infrastructure only (see the package docstring).

Field storage inside the oracle ("full" arrays, both walls stored):
    U  (nz, ny, nx+1)   x-velocity on x-faces x_f[0..nx]      (U[...,0] = U[...,nx] = 0)
    V  (nz, ny+1, nx)   y-velocity on y-faces                  (walls zero)
    W  (nz+1, ny, nx)   z-velocity on z-faces                  (walls zero)
    T  (nz, ny, nx)     temperature at cell centres
Exchange layout (the library's layout, see include/cube_fv.h): four (nz, ny, nx)
arrays; the face-normal velocity's slot i along its own axis is face i, so slot 0
is the wall at 0 and the wall at 1 is not stored.

Equations (Section 2, Eqs. 1-6) in the unit-viscosity form
    dv/dt = -div(v v) + Lap v + Gr T e_z - grad p ,   dT/dt = -div(v T) + Lap T / Pr ,  div v = 0
with no-slip walls, T = 1 at x = 0 and T = 0 at x = 1 (Eq. 4), dT/dy = 0 at
y = 0, 1 (Eq. 5) and dT/dz = 0 at z = 0, 1 (Eq. 6).  F excludes the pressure
gradient: the steady state solves P F(q) = 0 with D q = 0.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- grid
def faces(n: int, stretch: float) -> np.ndarray:
    """Face coordinates x_f[0..n] of one axis of [0,1].

    stretch == 0: uniform i/n.  Otherwise the tanh law
        x_f[i] = (1 + tanh(s (2 i / n - 1)) / tanh(s)) / 2,
    which clusters faces toward both walls (Section 4.1, "stretched near the
    borders"; the law and the factor s are this implementation's reading).  The
    lower half is computed and mirrored, x_f[n - i] = 1 - x_f[i], so the grid
    is exactly symmetric about 1/2 and the symmetries of Section 2 hold
    bit-for-bit on the index grid.
    """
    i = np.arange(n + 1, dtype=np.float64)
    if stretch == 0.0:
        xf = i / n
    else:
        xf = 0.5 * (1.0 + np.tanh(stretch * (2.0 * i / n - 1.0)) / np.tanh(stretch))
    half = n // 2
    for k in range(0, half + 1):
        xf[n - k] = 1.0 - xf[k]
    if n % 2 == 0:
        xf[half] = 0.5
    xf[0], xf[n] = 0.0, 1.0
    return xf


class Axis:
    """Metric arrays of one axis with n cells (faces from `faces(n, stretch)`, or the given xf)."""

    def __init__(self, n: int, stretch: float, xf=None):
        self.n = n
        if xf is None:
            self.xf = faces(n, stretch)
        else:
            self.xf = np.array(xf, dtype=np.float64)
            if self.xf.shape != (n + 1,) or self.xf[0] != 0.0 or self.xf[-1] != 1.0 or np.any(np.diff(self.xf) <= 0):
                raise ValueError("faces must be n + 1 strictly increasing values from 0 to 1")
        self.dx = np.diff(self.xf)                      # cell widths, n
        self.xc = 0.5 * (self.xf[:-1] + self.xf[1:])    # cell centres (face midpoints), n
        self.dc = np.diff(self.xc)                      # centre spacing across interior face i = 1..n-1, n-1
        # linear interpolation from centres i-1, i to interior face i (exact: centres are face midpoints)
        s = self.dx[:-1] + self.dx[1:]
        self.wl = self.dx[1:] / s                       # weight of cell i-1
        self.wr = self.dx[:-1] / s                      # weight of cell i


class Grid:
    """Tensor-product grid of the unit cube; axes[0] = x, axes[1] = y, axes[2] = z.  xyz_faces: optional
    (xf, yf, zf), each None (the stretch law) or the n + 1 faces of that axis."""

    def __init__(self, nx: int, ny: int, nz: int, stretch: float = 0.0, Pr: float = 0.71, xyz_faces=None):
        f = xyz_faces if xyz_faces is not None else (None, None, None)
        self.axes = [Axis(nx, stretch, f[0]), Axis(ny, stretch, f[1]), Axis(nz, stretch, f[2])]
        self.nx, self.ny, self.nz = nx, ny, nz
        self.Pr = Pr

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def full_shape(self, c: int):
        """Shape of the full (both walls) array of velocity component c (0 = u, 1 = v, 2 = w)."""
        s = [self.nz, self.ny, self.nx]
        s[2 - c] += 1
        return tuple(s)


# ----------------------------------------------------------------------------- helpers
def _sl(ax: int, s: slice):
    idx = [slice(None)] * 3
    idx[ax] = s
    return tuple(idx)


def _b(vec: np.ndarray, ax: int) -> np.ndarray:
    """Broadcast a 1D metric array along numpy axis ax (numpy axis of direction d is 2 - d)."""
    shape = [1, 1, 1]
    shape[ax] = vec.shape[0]
    return vec.reshape(shape)


def _interp_to_interior_faces(a: np.ndarray, g: Axis, ax: int) -> np.ndarray:
    """Cell values (n along ax) -> values on interior faces 1..n-1 (n-1 along ax)."""
    return _b(g.wl, ax) * a[_sl(ax, slice(0, -1))] + _b(g.wr, ax) * a[_sl(ax, slice(1, None))]


def _pad_walls(a: np.ndarray, ax: int) -> np.ndarray:
    """Interior-face values (n-1 along ax) -> all faces (n+1) with zeros on both walls."""
    pad = [(0, 0)] * 3
    pad[ax] = (1, 1)
    return np.pad(a, pad)


# ----------------------------------------------------------------------------- layout
def from_api(grid: Grid, q_api) -> list[np.ndarray]:
    """Exchange layout (four (nz,ny,nx) arrays) -> full arrays; wall slots are taken as zero."""
    out = []
    for c in range(3):
        ax = 2 - c
        a = np.asarray(q_api[c], dtype=np.float64)
        interior = a[_sl(ax, slice(1, None))]           # faces 1..n-1
        out.append(_pad_walls(interior, ax))
    out.append(np.array(q_api[3], dtype=np.float64))
    return out


def to_api(grid: Grid, q_full) -> list[np.ndarray]:
    """Full arrays -> exchange layout (slot i = face i; the wall at 1 is dropped)."""
    out = []
    for c in range(3):
        ax = 2 - c
        a = np.array(q_full[c][_sl(ax, slice(0, -1))], dtype=np.float64)
        a[_sl(ax, slice(0, 1))] = 0.0
        out.append(a)
    out.append(np.array(q_full[3], dtype=np.float64))
    return out


def interior_velocity(q_full, c: int) -> np.ndarray:
    return q_full[c][_sl(2 - c, slice(1, -1))]


def pack(q_full) -> np.ndarray:
    """Unknown vector: interior faces of u, v, w, then T, each C-ordered."""
    return np.concatenate([interior_velocity(q_full, c).ravel() for c in range(3)] + [q_full[3].ravel()])


def unpack(grid: Grid, x: np.ndarray) -> list[np.ndarray]:
    out, o = [], 0
    for c in range(3):
        s = list(grid.full_shape(c))
        s[2 - c] -= 2
        n = int(np.prod(s))
        out.append(_pad_walls(x[o:o + n].reshape(s), 2 - c))
        o += n
    out.append(x[o:o + grid.nx * grid.ny * grid.nz].reshape(grid.shape).copy())
    return out


def n_unknowns(grid: Grid) -> int:
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    return (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1) + nx * ny * nz


# ----------------------------------------------------------------------------- operators
def convection(grid: Grid, a, b):
    """Bilinear conservative convection div(a b) with advecting field a, advected field b.

    Returns the interior-face values for u, v, w (each with n_c - 1 slots along
    its own axis) and the cell values for T.  Momentum component c, direction d:
      d == c : flux on the c-CV faces (cell centres) = (mean a_c)(mean b_c), the
               means of the two neighbouring faces, then differenced over the
               centre spacing;
      d != c : flux on d-faces = a_d interpolated along c to the c-face, times
               b_c interpolated along d to the d-face (zero at a wall), then
               differenced over the cell width.
    Temperature: flux on d-faces = a_d times T interpolated to the face.  The
    advecting velocity is zero on every wall (no-slip / no penetration, Section 2).
    """
    ax_ = grid.axes
    out = []
    for c in range(3):
        axc = 2 - c
        gc = ax_[c]
        acc = None
        for d in range(3):
            axd = 2 - d
            gd = ax_[d]
            if d == c:
                am = 0.5 * (a[c][_sl(axc, slice(0, -1))] + a[c][_sl(axc, slice(1, None))])
                bm = 0.5 * (b[c][_sl(axc, slice(0, -1))] + b[c][_sl(axc, slice(1, None))])
                term = np.diff(am * bm, axis=axc) / _b(gc.dc, axc)
            else:
                ad_c = _interp_to_interior_faces(a[d], gc, axc)          # n_d+1 along d
                bc_i = b[c][_sl(axc, slice(1, -1))]                      # interior c-faces, cells along d
                bc_d = _pad_walls(_interp_to_interior_faces(bc_i, gd, axd), axd)
                term = np.diff(ad_c * bc_d, axis=axd) / _b(gd.dx, axd)
            acc = term if acc is None else acc + term
        out.append(acc)
    accT = None
    for d in range(3):
        axd = 2 - d
        gd = ax_[d]
        Td = _pad_walls(_interp_to_interior_faces(b[3], gd, axd), axd)
        term = np.diff(a[d] * Td, axis=axd) / _b(gd.dx, axd)
        accT = term if accT is None else accT + term
    out.append(accT)
    return out


def diffusion(grid: Grid, b, T_hot: float):
    """Lap of each velocity component (no-slip walls) and Lap T / Pr with Eqs. 4-6.

    Wall gradients use the half-cell distance from the first centre to the wall.
    T_hot is the Dirichlet value at x = 0 (1 in F, 0 in the linearisation);
    the value at x = 1 is 0 in both.
    """
    ax_ = grid.axes
    out = []
    for c in range(3):
        axc = 2 - c
        gc = ax_[c]
        acc = None
        for d in range(3):
            axd = 2 - d
            gd = ax_[d]
            if d == c:
                grad = np.diff(b[c], axis=axc) / _b(gc.dx, axc)          # at cell centres
                term = np.diff(grad, axis=axc) / _b(gc.dc, axc)
            else:
                bi = b[c][_sl(axc, slice(1, -1))]
                inner = np.diff(bi, axis=axd) / _b(gd.dc, axd)
                lo = (bi[_sl(axd, slice(0, 1))] - 0.0) / (0.5 * gd.dx[0])
                hi = (0.0 - bi[_sl(axd, slice(-1, None))]) / (0.5 * gd.dx[-1])
                grad = np.concatenate([lo, inner, hi], axis=axd)
                term = np.diff(grad, axis=axd) / _b(gd.dx, axd)
            acc = term if acc is None else acc + term
        out.append(acc)
    T = b[3]
    accT = None
    for d in range(3):
        axd = 2 - d
        gd = ax_[d]
        inner = np.diff(T, axis=axd) / _b(gd.dc, axd)
        if d == 0:   # Eq. 4: Dirichlet at x = 0 (T_hot) and x = 1 (0)
            lo = (T[_sl(axd, slice(0, 1))] - T_hot) / (0.5 * gd.dx[0])
            hi = (0.0 - T[_sl(axd, slice(-1, None))]) / (0.5 * gd.dx[-1])
        else:        # Eqs. 5-6: zero normal gradient
            lo = np.zeros_like(T[_sl(axd, slice(0, 1))])
            hi = np.zeros_like(lo)
        grad = np.concatenate([lo, inner, hi], axis=axd)
        term = np.diff(grad, axis=axd) / _b(gd.dx, axd)
        accT = term if accT is None else accT + term
    out.append(accT / grid.Pr)
    return out


def buoyancy(grid: Grid, T: np.ndarray, Gr: float) -> np.ndarray:
    """Gr T e_z on the interior z-faces, T interpolated linearly between the two centres."""
    return Gr * _interp_to_interior_faces(T, grid.axes[2], 0)


def _assemble(grid: Grid, parts):
    """Interior-face momentum parts + T part -> full arrays (walls zero)."""
    return [_pad_walls(parts[c], 2 - c) for c in range(3)] + [parts[3]]


def residual_full(grid: Grid, Gr: float, q):
    """F(q; Gr) = -div(v v) + Lap v + Gr T e_z (momentum), -div(v T) + Lap T / Pr (energy)."""
    C = convection(grid, q, q)
    L = diffusion(grid, q, 1.0)
    parts = [-C[c] + L[c] for c in range(4)]
    parts[2] = parts[2] + buoyancy(grid, q[3], Gr)
    return _assemble(grid, parts)


def jvp_full(grid: Grid, Gr: float, q, v):
    """J(q) v, the exact derivative of F at q along v.

    F is quadratic in q, so J(q) v = -div(q v) - div(v q) + Lap v + Gr T_v e_z,
    with the diffusion taken with homogeneous wall data (the Dirichlet value 1
    of Eq. 4 is part of F's constant term, not of J).
    """
    C1 = convection(grid, q, v)
    C2 = convection(grid, v, q)
    L = diffusion(grid, v, 0.0)
    parts = [-C1[c] - C2[c] + L[c] for c in range(4)]
    parts[2] = parts[2] + buoyancy(grid, v[3], Gr)
    return _assemble(grid, parts)


def divergence_full(grid: Grid, vel) -> np.ndarray:
    """(D v)_cell = sum_d (v_d(face+) - v_d(face-)) / width_d, wall fluxes zero (continuity, Eq. 3)."""
    acc = None
    for d in range(3):
        axd = 2 - d
        term = np.diff(vel[d], axis=axd) / _b(grid.axes[d].dx, axd)
        acc = term if acc is None else acc + term
    return acc


def gradient_full(grid: Grid, phi: np.ndarray):
    """(G phi)_face = (phi(cell+) - phi(cell-)) / centre spacing on interior faces, zero on walls."""
    out = []
    for c in range(3):
        axc = 2 - c
        out.append(_pad_walls(np.diff(phi, axis=axc) / _b(grid.axes[c].dc, axc), axc))
    return out


# ----------------------------------------------------------------------------- exchange-layout wrappers
def residual(grid: Grid, Gr: float, q_api):
    return to_api(grid, residual_full(grid, Gr, from_api(grid, q_api)))


def jvp(grid: Grid, Gr: float, q_api, v_api):
    return to_api(grid, jvp_full(grid, Gr, from_api(grid, q_api), from_api(grid, v_api)))


def conduction_state(grid: Grid):
    """u = 0, T = 1 - x_c: the exact steady state at Gr = 0 (full arrays)."""
    q = [np.zeros(grid.full_shape(c)) for c in range(3)]
    xc = grid.axes[0].xc
    q.append(np.broadcast_to(1.0 - xc[None, None, :], grid.shape).copy())
    return q
