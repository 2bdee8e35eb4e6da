"""Plain FP64 CPU oracle for the staggered finite-volume cube problem.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) may import, call, link or execute anything in this package.
Only the test-suite, the package's smoke check and the benchmark's CPU-baseline
leg use it.

What it computes (Gelfgat, "Sequence of bifurcations of natural convection of
air in a laterally heated cube ..."):

* Eqs. 1-3 (Boussinesq momentum, energy, continuity) with the boundary
  conditions of Eqs. 4-6, written in the unit-viscosity scaling
  ("Form A": velocity nu/H, time H^2/nu, pressure rho nu^2/H^2, buoyancy
  Gr*T*e_z, thermal diffusion 1/Pr).  The paper's Eqs. 1-2 use the extra
  Gr^(1/2) rescaling of Section 2; the two forms are related by
  v_A = Gr^(1/2) v_B, t_A = Gr^(-1/2) t_B, p_A = Gr p_B, so eigenvalues obey
  lambda_A = Gr^(1/2) lambda_B.  Form A stays regular at Gr = 0.
* The residual F(q; Gr), its Jacobian-vector product J(q) v, the discrete
  divergence D and gradient G, and the projection P = I - G (DG)^+ D that makes
  a velocity field discretely divergence-free (the "SIMPLE-like" divergence-free
  Krylov vectors of Section 1 / Section 3).
* Newton's method with BiCGstab(2) / GMRES inner solves and the Chebyshev-
  preconditioned Arnoldi iteration for the leading eigenvalues (Section 1,
  methods paragraph; Section 4.1 asks for four leading eigenvalues).
* The symmetry measures of Eqs. 7-9 and the diagnostics of Eqs. 12-13.

The discretisation itself is not printed in the paper (Section 3 defers to its
refs. 14-16); the readings used here are: MAC staggering, conservative central
fluxes with linear interpolation, half-cell wall distances, and a tanh grid
stretched symmetrically toward every wall (Section 4.1: "stretched near the
borders").

Parity status: every function here is pinned by tests under tests/ against
closed forms, exact invariants, manufactured solutions or library routines,
except where a docstring says "parity unpinned".
"""
