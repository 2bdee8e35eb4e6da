"""Divergence-free projection P = I - G (DG)^+ D of the velocity part (FP64, numpy).

Test infrastructure only (see the package docstring).

Section 1 (methods paragraph) and Section 3: every Krylov vector is made
divergence free and consistent with the boundary conditions by a SIMPLE-like
pressure correction.  The reading taken here is the exact projector onto
null(D) along range(G): solve the cell-centred Neumann problem DG phi = D v and
correct v <- v - G phi.  Temperature passes through unchanged.

Poisson solver: fast diagonalisation (Lynch, Rice & Thomas 1964).  DG is the
Kronecker sum A_x (+) A_y (+) A_z of 1D operators A = diag(1/width) S with S
symmetric tridiagonal, so with the generalised eigenvectors S e = lam diag(width) e
    phi = (E_z x E_y x E_x) diag(1/(lam_x + lam_y + lam_z)) (E_z x E_y x E_x)^-1 rhs,
the constant (zero-eigenvalue) mode set to zero.  A conjugate-gradient solve
is kept beside it as an independent cross-check.
"""
from __future__ import annotations

import numpy as np

from .discretisation import Axis, Grid, divergence_full, gradient_full, from_api, to_api


def neumann_matrix(g: Axis) -> np.ndarray:
    """Dense 1D operator (A phi)_i = (flux_{i+1} - flux_i) / width_i, flux_i = (phi_i - phi_{i-1}) / spacing_i,
    with zero flux through both walls."""
    n = g.n
    A = np.zeros((n, n))
    for i in range(n):
        if i + 1 <= n - 1:
            c = 1.0 / g.dc[i]          # face i+1 has spacing dc[i]
            A[i, i + 1] += c / g.dx[i]
            A[i, i] -= c / g.dx[i]
        if i >= 1:
            c = 1.0 / g.dc[i - 1]      # face i
            A[i, i - 1] += c / g.dx[i]
            A[i, i] -= c / g.dx[i]
    return A


class FDM:
    """Fast-diagonalisation solver of DG phi = rhs on a Grid."""

    def __init__(self, grid: Grid):
        self.grid = grid
        self.lam, self.E, self.Einv = [], [], []
        for g in grid.axes:
            A = neumann_matrix(g)
            sq = np.sqrt(g.dx)
            B = (sq[:, None] * A) / sq[None, :]          # diag(w^1/2) A diag(w^-1/2), symmetric
            B = 0.5 * (B + B.T)
            lam, Y = np.linalg.eigh(B)
            self.lam.append(lam)
            self.E.append(Y / sq[:, None])               # E = W^-1/2 Y
            self.Einv.append(Y.T * sq[None, :])          # E^-1 = Y^T W^1/2
        lx, ly, lz = self.lam
        self.den = lz[:, None, None] + ly[None, :, None] + lx[None, None, :]
        self.zero = np.unravel_index(np.argmax(self.den), self.den.shape)   # the constant mode (lam = 0)

    def _apply(self, M, a, axis):
        # contract axis `axis` (numpy) of a with the columns of M: out[..m..] = sum_i M[m, i] a[..i..]
        return np.moveaxis(np.tensordot(M, a, axes=([1], [axis])), 0, axis)

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        Ex, Ey, Ez = self.E
        Ix, Iy, Iz = self.Einv
        h = self._apply(Ix, rhs, 2)
        h = self._apply(Iy, h, 1)
        h = self._apply(Iz, h, 0)
        den = self.den.copy()
        den[self.zero] = 1.0
        h = h / den
        h[self.zero] = 0.0
        h = self._apply(Ex, h, 2)
        h = self._apply(Ey, h, 1)
        h = self._apply(Ez, h, 0)
        return h


def laplacian(grid: Grid, phi: np.ndarray) -> np.ndarray:
    return divergence_full(grid, gradient_full(grid, phi))


def cg_solve(grid: Grid, rhs: np.ndarray, tol: float = 1e-14, max_it: int = 20000) -> np.ndarray:
    """Conjugate gradients on -DG phi = -rhs in the cell-volume inner product.

    DG is self-adjoint and negative semi-definite in <a, b> = sum V_c a_c b_c;
    rhs (a divergence) has zero volume-weighted mean, so CG stays in the
    complement of the constants.
    """
    gx, gy, gz = grid.axes
    V = gz.dx[:, None, None] * gy.dx[None, :, None] * gx.dx[None, None, :]
    dot = lambda a, b: float(np.sum(V * a * b))
    b = -rhs - dot(-rhs, np.ones_like(rhs)) / float(V.sum())
    x = np.zeros_like(rhs)
    r = b.copy()
    p = r.copy()
    rr = dot(r, r)
    r0 = np.sqrt(rr)
    for _ in range(max_it):
        if np.sqrt(rr) <= tol * r0:
            break
        Ap = -laplacian(grid, p)
        alpha = rr / dot(p, Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = dot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


class Projector:
    """P on full arrays (velocity projected, T unchanged) and on the exchange layout."""

    def __init__(self, grid: Grid, solver: str = "fdm"):
        self.grid = grid
        self.solver = solver
        self.fdm = FDM(grid) if solver == "fdm" else None

    def potential(self, vel) -> np.ndarray:
        rhs = divergence_full(self.grid, vel)
        if self.solver == "fdm":
            return self.fdm.solve(rhs)
        return cg_solve(self.grid, rhs)

    def full(self, q):
        phi = self.potential(q[:3])
        G = gradient_full(self.grid, phi)
        out = [q[c] - G[c] for c in range(3)]
        out.append(np.array(q[3], dtype=np.float64, copy=True) if len(q) > 3 else None)
        return out if len(q) > 3 else out[:3]

    def api(self, q_api):
        return to_api(self.grid, self.full(from_api(self.grid, q_api)))
