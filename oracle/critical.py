"""Critical Grashof number of one grid by bisection (FP64, scipy).

Test infrastructure only (see the package docstring).  Section 4.1 locates, on each grid, the Gr at which
the real part of a leading eigenvalue of the linearised problem crosses zero (then extrapolates those to
zero grid size, Table 1).  Here, plainly: the symmetric steady state (the flows below the first bifurcations keep the three
symmetries of Section 2) by Newton with sparse-LU corrections, symmetrised after every step
(sparse.newton_direct), the eigenvalues nearest the given shifts by ARPACK shift-invert on the saddle
pencil (sparse.shift_invert_eigs), the tracked one (largest real part overall, among real values, or
among complex pairs), and bisection of a bracketing interval until it is tol relative wide.
"""
from __future__ import annotations

import numpy as np

from . import discretisation as D
from . import sparse as S


def tracked(lam, mode: str):
    """The eigenvalue of largest real part among all ('leading'), the real ('real') or the complex
    ('oscillatory', +Im member) values."""
    cand = [z for z in lam
            if mode == "leading" or (mode == "real" and z.imag == 0.0) or (mode == "oscillatory" and z.imag > 0.0)]
    if not cand:
        raise ValueError("no eigenvalue of the tracked kind: add shifts or raise k")
    return max(cand, key=lambda z: z.real)


def critical_gr(grid: D.Grid, gr_lo: float, gr_hi: float, q_lo, mode: str, shifts, k=8, tol=1e-9):
    """Bisection on Re lam(Gr) over [gr_lo, gr_hi] (signs must differ).  q_lo: a steady state at or near
    gr_lo (full arrays).  Returns (gr_cr, lam at the last midpoint, history [(gr, lam)])."""
    hist = []

    def f(gr, q):
        q, rep = S.newton_direct(grid, gr, q, tol=1e-10, max_newton=25, atol=1e-5, symmetric=True)
        if rep["status"] != "converged":
            raise RuntimeError(f"Newton did not converge at Gr = {gr}")
        lam = tracked(S.shift_invert_eigs(grid, gr, q, shifts, k=k), mode)
        hist.append((gr, lam))
        return lam, q

    la, qa = f(gr_lo, q_lo)
    lb, qb = f(gr_hi, qa)
    if la.real * lb.real > 0.0:
        raise ValueError("the interval does not bracket a crossing")
    lo, hi, lam = gr_lo, gr_hi, lb
    while (hi - lo) > tol * hi:
        mid = 0.5 * (lo + hi)
        lam, qm = f(mid, qa)
        if lam.real * la.real > 0.0:
            lo, la, qa = mid, lam, qm
        else:
            hi = mid
    return 0.5 * (lo + hi), lam, hist
