"""Semi-implicit time step of the full equations (FP64, numpy + scipy sparse LU).

Test infrastructure only (see the package docstring).  Section 4.2.3 integrates Eqs. 1-6 in time at slightly
sub- and supercritical Gr and follows the kinetic energy (Eq. 12) and the hot-wall Nusselt number (Eq. 13).
The step written out here, the plain definition of the library's scheme:

    (I - dt L) delta = dt F(q_n; Gr),   q_{n+1} = q_n + P delta,

with L the diffusion part of J (the Laplacian of every velocity component with no-slip walls, Lap T / Pr
with homogeneous Eqs. 4-6: F carries the Dirichlet data) assembled as a sparse matrix and factorised, F the
residual of discretisation.py, and P the projection of projection.py acting on the velocity part.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import discretisation as D
from . import diagnostics as DG
from . import sparse as S
from .projection import Projector


def diffusion_matrix(grid: D.Grid) -> sp.csr_matrix:
    """L on the packed unknowns (homogeneous wall data), assembled by probing D.diffusion."""
    shapes = S._block_shapes(grid)

    def apply(x):
        parts = D.diffusion(grid, D.unpack(grid, x), 0.0)
        full = [D._pad_walls(parts[c], 2 - c) for c in range(3)] + [parts[3]]
        return D.pack(full)

    return S._probe(apply, shapes, shapes)


class SemiImplicit:
    """Steps of size dt at Gr on one grid (the factorisation of I - dt L is kept)."""

    def __init__(self, grid: D.Grid, Gr: float, dt: float):
        self.grid, self.Gr, self.dt = grid, Gr, dt
        n = D.n_unknowns(grid)
        self.lu = spla.splu((sp.identity(n) - dt * diffusion_matrix(grid)).tocsc())
        self.P = Projector(grid)

    def step(self, q):
        F = D.pack(D.residual_full(self.grid, self.Gr, q))
        delta = D.unpack(self.grid, self.lu.solve(self.dt * F))
        delta = self.P.full(delta)
        return [q[c] + delta[c] for c in range(4)]

    def run(self, q, nsteps):
        """q after nsteps steps, and the (E_kin, Nu) histories before the first and after every step."""
        ek, nu = [DG.kinetic_energy(self.grid, q)], [DG.nusselt_hot(self.grid, q[3])]
        for _ in range(nsteps):
            q = self.step(q)
            ek.append(DG.kinetic_energy(self.grid, q))
            nu.append(DG.nusselt_hot(self.grid, q[3]))
        return q, np.array(ek), np.array(nu)
