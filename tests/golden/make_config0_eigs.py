"""Writes config0_eigs_32.txt: the oracle's leading eigenvalues for the 32^3 uniform cube at Gr = 1e5.

Pr = 0.71; steady state by the oracle's Newton method (continuation 1.25e4 -> 1e5 in x2 steps,
tol 1e-11); four leading eigenvalues of P J by the oracle's Chebyshev-preconditioned Arnoldi (m = 20,
residual tol 1e-9).  Calls only oracle/ (and numpy); takes ~15 minutes on one CPU core.
Run:  python tests/golden/make_config0_eigs.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.discretisation as D  # noqa: E402
from oracle import solvers as SV  # noqa: E402


def main():
    n, Gr, Pr = 32, 1.0e5, 0.71
    g = D.Grid(n, n, n, stretch=0.0, Pr=Pr)
    q = D.conduction_state(g)
    G = 1.25e4
    while True:
        q, rep = SV.newton_steady(g, min(G, Gr), q, tol=1e-11, max_matvec=6000)
        assert rep["status"] == "converged", rep
        if G >= Gr:
            break
        G *= 2.0
    x0 = np.random.default_rng(3).standard_normal(D.n_unknowns(g))
    lam, _, info = SV.leading_eigenvalues(g, Gr, q, k=4, m=20, seed_vector=x0, tol=1e-9)
    assert info["converged"], info
    out = os.path.join(HERE, "config0_eigs_32.txt")
    with open(out, "w") as f:
        f.write("# Oracle leading eigenvalues (Form A units), 32^3 uniform cube, Pr = 0.71, Gr = 1e5.\n")
        f.write("# Written by tests/golden/make_config0_eigs.py (oracle Newton + Chebyshev-Arnoldi, tol 1e-9).\n")
        f.write(f"# restarts {info['restarts']}, matvecs {info['matvecs']}, residuals {list(info['residual'])}\n")
        for z in lam:
            f.write(f"{z.real:.15e} {z.imag:.15e}\n")
    print(out)


if __name__ == "__main__":
    main()
