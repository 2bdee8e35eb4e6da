"""Writes tests/golden/critical_gr_12_pr0.015.txt: the critical Gr of the steady (real) and of the
oscillatory mode on a 12^3 tanh-stretched grid (s = 1.5) at Pr = 0.015, where both cross between
Gr = 3.9e5 and 4.4e5 (Section 4.1 finds two modes crossing at close Gr; this coarse grid at a low Prandtl
number puts such a pair within reach of the oracle).  Calls only oracle/: the steady state along a Gr
ladder by oracle.sparse.newton_direct, then oracle.critical.critical_gr (bisection to 1e-9 relative,
eigenvalues by ARPACK shift-invert near the shifts 5 and 5 + 480i).  About 30 minutes on 8 cores.

    python tests/golden/make_critical_gr.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle.discretisation as D  # noqa: E402
from oracle import critical as CR  # noqa: E402
from oracle import sparse as S  # noqa: E402

N, STRETCH, PR = 12, 1.5, 0.015
LO, HI = 3.9e5, 4.4e5
SHIFTS = [5.0, 5.0 + 480j]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "critical_gr_12_pr0.015.txt")


def main():
    g = D.Grid(N, N, N, stretch=STRETCH, Pr=PR)
    q = D.conduction_state(g)
    gr = 1.25e4
    while gr < LO:
        q, rep = S.newton_direct(g, gr, q, tol=1e-10, max_newton=25)
        print(f"Gr {gr:.4g}: {rep['status']}", flush=True)
        gr = min(2.0 * gr, LO)
    q, _ = S.newton_direct(g, LO, q, tol=1e-10, max_newton=25, atol=1e-5)
    rows = []
    for mode in ("real", "oscillatory"):
        gcr, lam, hist = CR.critical_gr(g, LO, HI, q, mode, SHIFTS, k=8, tol=1e-9)
        print(mode, gcr, lam, flush=True)
        rows.append((mode, gcr, lam))
    with open(OUT, "w") as f:
        f.write(f"# critical Gr, {N}^3 tanh-stretched s = {STRETCH}, Pr = {PR} (Form A eigenvalues)\n")
        f.write("# oracle: sparse-LU Newton, ARPACK shift-invert near 5 and 5+480i, bisection to 1e-9\n")
        f.write("# mode gr_cr re_lam im_lam\n")
        for mode, gcr, lam in rows:
            f.write(f"{mode} {gcr:.12e} {lam.real:.6e} {abs(lam.imag):.12e}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
