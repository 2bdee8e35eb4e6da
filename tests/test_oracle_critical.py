"""Pin of the stored critical Grashof numbers (tests/golden/critical_gr_12_pr0.015.txt) against their
definition (Section 4.1): the real part of the tracked eigenvalue of the linearised problem about the
steady state has opposite signs 1e-4 (relative) below and above Gr_cr, and the line through those two
values crosses zero at Gr_cr to 1e-6.  The steady state
and the eigenvalues are recomputed here along the oracle's sparse path (a Gr ladder of sparse-LU Newton
solves, ARPACK shift-invert), about two minutes.
"""
import os

import pytest

import oracle.discretisation as D
from oracle import critical as CR
from oracle import sparse as S

N, STRETCH, PR = 12, 1.5, 0.015
SHIFTS = [5.0, 5.0 + 480j]


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "critical_gr_12_pr0.015.txt")
    rows = {}
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            mode, gcr, lr, li = ln.split()
            rows[mode] = (float(gcr), float(lr), float(li))
    return rows


def test_stored_critical_values_satisfy_the_definition():
    g = D.Grid(N, N, N, stretch=STRETCH, Pr=PR)
    q = D.conduction_state(g)
    for gr in (1.25e4, 5e4, 2e5, 3.9e5):
        q, rep = S.newton_direct(g, gr, q, tol=1e-10, max_newton=25, atol=1e-5)
        assert rep["status"] == "converged", gr
    shift = {"real": [5.0], "oscillatory": [5.0 + 480j]}
    for mode, (gcr, _, im_ref) in sorted(_golden().items()):
        lams = []
        for x in (gcr * (1 - 1e-4), gcr * (1 + 1e-4)):
            qx, rep = S.newton_direct(g, x, q, tol=1e-10, max_newton=25, atol=1e-5, symmetric=True)
            assert rep["status"] == "converged"
            lams.append(CR.tracked(S.shift_invert_eigs(g, x, qx, shift[mode], k=6), mode))
        lo, hi = lams
        # the real part changes sign across Gr_cr (1e-4 relative either side)
        assert lo.real < 0.0 < hi.real or hi.real < 0.0 < lo.real, (mode, lo, hi)
        # and Gr_cr sits where the line through the two values crosses zero, to 1e-6 relative
        x0 = gcr * (1 - 1e-4) - lo.real * (2e-4 * gcr) / (hi.real - lo.real)
        assert abs(x0 - gcr) <= 1e-6 * gcr, (mode, x0, gcr)
        if mode == "oscillatory":
            assert abs(0.5 * (lo.imag + hi.imag)) == pytest.approx(im_ref, rel=1e-5)
