"""Sparse assembly of the discrete operators, direct Newton and shift-invert eigenvalues (FP64, scipy).

Test infrastructure only (see the package docstring).  An eigen-solver that shares nothing with the
library's Krylov methods (no Chebyshev filter, no implicit-Euler transform, no GMRES): the leading
eigenvalues of the linearised problem (Section 1 methods paragraph, Section 4.1)

    lambda v = J(q) v - G p,   D v = 0

are the finite eigenvalues of the sparse pencil (A, B),

    A = [[J, -G], [D, 0]],   B = [[I, 0], [0, 0]]      (unknowns: v and T, then p),

which this module builds explicitly and hands to a sparse LU factorisation and ARPACK in shift-invert
mode.  The pressure's constant mode (G 1 = 0) and the matching dependent divergence row (the volume-
weighted sum of D v vanishes for no-through-flow walls) are removed by dropping pressure unknown 0 and
divergence row 0, which leaves a regular pencil with the same finite eigenvalues.

Every matrix is assembled by probing the oracle's matrix-free operators (discretisation.py) with sums
of unit vectors that share no output row: every coupling of this stencil connects unknowns at most one
index apart along each axis (the staggered offsets included), so unknowns of one field whose indices agree
modulo 3 along every axis (a colour) touch disjoint rows, and the unknown behind a row's entry is the one
of that colour within one index of the row.  The tests check the assembled matrices against the
matrix-free products (a longer coupling would alias and fail them).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import discretisation as D

_PERIOD = 3


def _block_shapes(grid: D.Grid):
    """Shapes of the packed unknown blocks: interior u, v, w faces, then T (pack() order)."""
    shapes = []
    for c in range(3):
        s = list(grid.full_shape(c))
        s[2 - c] -= 2
        shapes.append(tuple(s))
    shapes.append(grid.shape)
    return shapes


def _positions(shapes):
    """(k, j, i) of every packed entry of the given blocks, and each block's offset."""
    ks, js, is_, offs, o = [], [], [], [], 0
    for s in shapes:
        k, j, i = np.indices(s)
        ks.append(k.ravel())
        js.append(j.ravel())
        is_.append(i.ravel())
        offs.append(o)
        o += int(np.prod(s))
    return np.concatenate(ks), np.concatenate(js), np.concatenate(is_), offs, o


def _probe(apply, in_shapes, out_shapes):
    """Sparse matrix of the linear map `apply` (packed input of in_shapes -> packed output of out_shapes)."""
    _, _, _, in_off, n_in = _positions(in_shapes)
    K, J, I, _, n_out = _positions(out_shapes)
    rows, cols, vals = [], [], []
    for b, s in enumerate(in_shapes):
        kb, jb, ib = np.indices(s)
        for a in itertools.product(range(_PERIOD), repeat=3):
            mask = (kb % _PERIOD == a[0]) & (jb % _PERIOD == a[1]) & (ib % _PERIOD == a[2])
            if not mask.any():
                continue
            x = np.zeros(n_in)
            x[in_off[b] + np.flatnonzero(mask)] = 1.0
            y = apply(x)
            r = np.flatnonzero(y)
            if r.size == 0:
                continue
            idx = []
            for pos, res, n in ((K[r], a[0], s[0]), (J[r], a[1], s[1]), (I[r], a[2], s[2])):
                d = (res - pos) % _PERIOD
                d = np.where(d > _PERIOD // 2, d - _PERIOD, d)
                idx.append(pos + d)
            ok = (idx[0] >= 0) & (idx[0] < s[0]) & (idx[1] >= 0) & (idx[1] < s[1]) & (idx[2] >= 0) & (idx[2] < s[2])
            if not np.all(ok):
                raise AssertionError("a coupling reaches further than the colouring allows")
            c = in_off[b] + np.ravel_multi_index(tuple(idx), s)
            rows.append(r)
            cols.append(c)
            vals.append(y[r])
    rows, cols, vals = (np.concatenate(a) if a else np.zeros(0) for a in (rows, cols, vals))
    return sp.csr_matrix((vals, (rows.astype(np.int64), cols.astype(np.int64))), shape=(n_out, n_in))


def jacobian(grid: D.Grid, Gr: float, q) -> sp.csr_matrix:
    """J(q) on the packed unknowns (interior u, v, w, then T)."""
    shapes = _block_shapes(grid)
    return _probe(lambda x: D.pack(D.jvp_full(grid, Gr, q, D.unpack(grid, x))), shapes, shapes)


def divergence(grid: D.Grid) -> sp.csr_matrix:
    """D: packed interior velocities -> cells."""
    vs = _block_shapes(grid)[:3]

    def apply(x):
        full = D.unpack(grid, np.concatenate([x, np.zeros(grid.nx * grid.ny * grid.nz)]))
        return D.divergence_full(grid, full[:3]).ravel()

    return _probe(apply, vs, [grid.shape])


def gradient(grid: D.Grid) -> sp.csr_matrix:
    """G: cells -> packed interior velocities."""
    vs = _block_shapes(grid)[:3]

    def apply(x):
        g = D.gradient_full(grid, x.reshape(grid.shape))
        return np.concatenate([D.interior_velocity(g, c).ravel() for c in range(3)])

    return _probe(apply, [grid.shape], vs)


def _constraint_blocks(grid: D.Grid):
    """-G and D padded to the packed unknowns (T has no pressure coupling), pressure 0 / row 0 removed."""
    n = D.n_unknowns(grid)
    Dm = divergence(grid)[1:, :]
    Gm = gradient(grid)[:, 1:]
    nv, npres = Dm.shape[1], Dm.shape[0]
    Gfull = sp.vstack([Gm, sp.csr_matrix((n - nv, npres))])
    Dfull = sp.hstack([Dm, sp.csr_matrix((npres, n - nv))])
    return Gfull, Dfull, npres


def symmetrise(q):
    """Mean of q over the symmetry group of Section 2 (identity, reflection y -> 1-y, rotation about
    x = z = 1/2, centro-symmetry; T maps affinely).  The symmetric steady states are its fixed points."""
    from .diagnostics import sym_2d, sym_3d, sym_ref
    imgs = [q, sym_ref(q), sym_2d(q), sym_3d(q)]
    return [sum(im[c] for im in imgs) / 4.0 for c in range(4)]


def newton_direct(grid: D.Grid, Gr: float, q0, tol=1e-11, max_newton=30, atol=0.0, symmetric=False):
    """Steady state of Eqs. 1-6 by Newton's method with exact (sparse LU) corrections:
        [[J(q), -G], [D, 0]] [delta; p] = [-F(q); 0],   q <- q + delta.
    q0 (full arrays) must be divergence free; every delta is, so q stays so.  The residual is the
    projected one, P F = F - G p with D (F - G p) = 0; stop when ||P F||_inf <= tol max(1, ||P F(q0)||_inf)
    or ||P F||_inf <= atol (a start that is already a steady state cannot gain a factor tol on its
    round-off level residual).  symmetric: every iterate is symmetrised (the branch of symmetric states,
    on which a symmetry-breaking eigenvalue crossing zero leaves the Jacobian regular).
    Returns (q, report)."""
    q = [a.copy() for a in q0]
    n = D.n_unknowns(grid)
    Gfull, Dfull, npres = _constraint_blocks(grid)
    proj = spla.splu(sp.bmat([[sp.identity(n), -Gfull], [Dfull, None]], format="csc"))
    hist = []
    for it in range(max_newton + 1):
        F = D.pack(D.residual_full(grid, Gr, q))
        PF = proj.solve(np.concatenate([F, np.zeros(npres)]))[:n]
        rn = float(np.max(np.abs(PF)))
        hist.append(rn)
        if rn <= tol * max(1.0, hist[0]) or rn <= atol:
            return q, {"status": "converged", "residual": hist, "steps": it}
        if it == max_newton:
            break
        K = sp.bmat([[jacobian(grid, Gr, q), -Gfull], [Dfull, None]], format="csc")
        delta = spla.splu(K).solve(np.concatenate([-F, np.zeros(npres)]))[:n]
        dq = D.unpack(grid, delta)
        # damping: the first of 1, 1/2, .., 1/64 of the correction that lowers ||P F||_inf
        lam = 1.0
        for _ in range(7):
            qt = [q[c] + lam * dq[c] for c in range(4)]
            if symmetric:  # near a symmetry-breaking crossing dq carries a large antisymmetric part
                qt = symmetrise(qt)
            with np.errstate(all="ignore"):
                Ft = D.pack(D.residual_full(grid, Gr, qt))
            if np.all(np.isfinite(Ft)):
                rt = float(np.max(np.abs(proj.solve(np.concatenate([Ft, np.zeros(npres)]))[:n])))
                if rt < rn:
                    break
            lam *= 0.5
        q = qt
    return q, {"status": "max_newton", "residual": hist, "steps": max_newton}


def saddle_pencil(grid: D.Grid, Gr: float, q):
    """(A, B) of the pencil above, CSC, with pressure unknown 0 and divergence row 0 removed."""
    Jm = jacobian(grid, Gr, q)
    Gfull, Dfull, npres = _constraint_blocks(grid)
    n = Jm.shape[0]
    A = sp.bmat([[Jm, -Gfull], [Dfull, None]], format="csc")
    B = sp.block_diag([sp.identity(n), sp.csr_matrix((npres, npres))], format="csc")
    return A, B


def shift_invert_eigs(grid: D.Grid, Gr: float, q, shifts, k=10, tol=1e-13):
    """Eigenvalues of the pencil nearest each shift (ARPACK on (A - s B)^-1 B), merged and ordered by real
    part descending (then |Im| descending, +Im first).  Duplicates found from several shifts are merged
    (relative distance below 1e-8)."""
    A, B = saddle_pencil(grid, Gr, q)
    found = []
    for s in shifts:
        M = (A - s * B).tocsc()
        if np.iscomplexobj(s) or isinstance(s, complex):
            M = M.astype(np.complex128)
        lu = spla.splu(M)
        n = A.shape[0]
        dt = np.complex128 if M.dtype == np.complex128 else np.float64
        op = spla.LinearOperator((n, n), matvec=lambda x, lu=lu: lu.solve(B @ x), dtype=dt)
        nu = spla.eigs(op, k=k, which="LM", tol=tol, return_eigenvectors=False,
                       v0=np.ones(n, dtype=dt) / np.sqrt(n))
        lam = s + 1.0 / nu
        for z in lam:
            if not any(abs(z - w) <= 1e-8 * max(1.0, abs(w)) for w in found):
                found.append(complex(z))
    lam = np.array(found)
    # a real pencil: conjugate pairs; return values with |Im| below round-off as real
    lam = np.where(np.abs(lam.imag) <= 1e-10 * np.abs(lam), lam.real + 0j, lam)
    order = sorted(range(len(lam)), key=lambda i: (-lam[i].real, -abs(lam[i].imag), -lam[i].imag))
    return lam[order]
