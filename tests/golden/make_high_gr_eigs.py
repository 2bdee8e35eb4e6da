"""Writes tests/golden/eigs_16_stretched_gr1.6e6.txt: the leading eigenvalues of the linearised problem
(Section 1 methods paragraph; Section 4.1 follows four of them) about the steady state of a 16^3 tanh-
stretched grid (s = 1.5) at Gr = 1.6e6, Pr = 0.71.

Calls only oracle/: the steady state by Newton's method with exact sparse-LU corrections along a Gr ladder
(x2 from 1.25e4, oracle.sparse.newton_direct), then the eigenvalues of the pencil [[J, -G], [D, 0]] /
[[I, 0], [0, 0]] nearest several shifts by ARPACK in shift-invert mode (oracle.sparse.shift_invert_eigs):
on the real axis right of the spectrum and at 10 +- i w for w up to 2000, so that no eigenvalue of large
imaginary part with a real part among the leading ones is missed.  About 15 minutes on 8 cores.

    python tests/golden/make_high_gr_eigs.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle.discretisation as D  # noqa: E402
from oracle import sparse as S  # noqa: E402

N, STRETCH, PR, GR = 16, 1.5, 0.71, 1.6e6
SHIFTS = [10.0, 10.0 + 250j, 10.0 + 500j, 10.0 + 1000j, 10.0 + 2000j]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "eigs_16_stretched_gr1.6e6.txt")


def main():
    g = D.Grid(N, N, N, stretch=STRETCH, Pr=PR)
    q = D.conduction_state(g)
    gr = 1.25e4
    while True:
        gr = min(gr, GR)
        q, rep = S.newton_direct(g, gr, q, tol=1e-11)
        print(f"Gr {gr:.4g}: {rep['status']} after {rep['steps']} steps, ||PF|| {rep['residual'][-1]:.3e}", flush=True)
        if rep["status"] != "converged":
            raise SystemExit("Newton did not converge")
        if gr >= GR:
            break
        gr *= 2.0
    lam = S.shift_invert_eigs(g, GR, q, SHIFTS, k=16)
    # the conjugate partner of a shift with +Im is implied; keep the values with Im >= 0 and add mirrors
    full = []
    for z in lam:
        full.append(z)
        if abs(z.imag) > 0 and not any(abs(w - np.conj(z)) <= 1e-8 * abs(z) for w in lam):
            full.append(np.conj(z))
    full = sorted(full, key=lambda z: (-z.real, -abs(z.imag), -z.imag))
    with open(OUT, "w") as f:
        f.write(f"# leading eigenvalues (Form A), {N}^3 tanh-stretched s = {STRETCH}, Pr = {PR}, Gr = {GR:g}\n")
        f.write("# oracle: Newton with sparse-LU corrections, ARPACK shift-invert on the saddle pencil\n")
        f.write(f"# shifts: {SHIFTS}\n")
        for z in full[:8]:
            f.write(f"{z.real:.15e} {z.imag:.15e}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
