"""Pins of the oracle's sparse path (oracle/sparse.py): assembled operators, direct Newton, and the
shift-invert eigen-solver that shares nothing with the library's Krylov methods.

* The assembled J(q), D and G equal the matrix-free oracle products on random vectors (a coupling longer
  than the probing colours allow would alias and fail this).
* Newton with sparse-LU corrections reaches the state of the Krylov Newton (tests pin that one to
  quadratic convergence and P F = 0), keeps D q = 0 and the three symmetries (Eqs. 7-9).
* The shift-invert eigenvalues of the saddle pencil equal numpy's dense eigen-solve of Z^T (P J) Z at
  Gr > 0, and the closed-form temperature spectrum at Gr = 0.
"""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle import diagnostics as DG
from oracle import solvers as SV
from oracle import sparse as S
from paper_2210_08816_gb300 import seeded

PR = 0.71


def _random_state(g, seed, sigma=0.7):
    q = D.from_api(g, seeded.normal_fields(seed, g.shape, sigma))
    q[3] = q[3] + (1.0 - g.axes[0].xc)[None, None, :]
    return q


def test_assembled_operators_equal_the_matrix_free_ones():
    g = D.Grid(7, 6, 5, stretch=1.5, Pr=PR)
    q = _random_state(g, 3)
    Gr = 3.0e4
    Jm, Dm, Gm = S.jacobian(g, Gr, q), S.divergence(g), S.gradient(g)
    rng = np.random.default_rng(1)
    n = D.n_unknowns(g)
    nv = n - g.nx * g.ny * g.nz
    for _ in range(3):
        x = rng.standard_normal(n)
        ref = D.pack(D.jvp_full(g, Gr, q, D.unpack(g, x)))
        assert np.max(np.abs(Jm @ x - ref)) <= 1e-13 * np.max(np.abs(ref))
        vel = D.unpack(g, np.concatenate([x[:nv], np.zeros(n - nv)]))[:3]
        ref = D.divergence_full(g, vel).ravel()
        assert np.max(np.abs(Dm @ x[:nv] - ref)) <= 1e-13 * np.max(np.abs(ref))
        phi = rng.standard_normal(g.nx * g.ny * g.nz)
        gf = D.gradient_full(g, phi.reshape(g.shape))
        ref = np.concatenate([D.interior_velocity(gf, c).ravel() for c in range(3)])
        assert np.max(np.abs(Gm @ phi - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_direct_newton_matches_krylov_newton():
    g = D.Grid(8, 7, 6, stretch=1.5, Pr=PR)
    Gr = 1.2e4
    q_k, rep_k = SV.newton_steady(g, Gr, D.conduction_state(g), tol=1e-11)
    q_d, rep_d = S.newton_direct(g, Gr, D.conduction_state(g), tol=1e-12)
    assert rep_k["status"] == "converged" and rep_d["status"] == "converged"
    scale = max(float(np.max(np.abs(a))) for a in q_k)
    assert max(float(np.max(np.abs(q_d[c] - q_k[c]))) for c in range(4)) <= 1e-9 * scale
    assert np.max(np.abs(D.divergence_full(g, q_d[:3]))) <= 1e-10 * scale / 0.01
    assert max(DG.symmetry_measures(g, q_d[3])) <= 1e-9


def test_shift_invert_matches_dense_eigensolve():
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_oracle_solvers import _dense_restricted
    g = D.Grid(8, 7, 6, stretch=1.5, Pr=PR)
    Gr = 1.2e4
    q, _ = S.newton_direct(g, Gr, D.conduction_state(g), tol=1e-12)
    lam_dense, _ = _dense_restricted(g, Gr, q)
    lam = S.shift_invert_eigs(g, Gr, q, [10.0], k=10)
    assert np.allclose(lam[:6], lam_dense[:6], rtol=1e-10, atol=0), (lam[:6], lam_dense[:6])


def test_shift_invert_gr0_closed_form():
    g = D.Grid(10, 8, 6, stretch=0.0, Pr=PR)
    lam = S.shift_invert_eigs(g, 0.0, D.conduction_state(g), [10.0], k=8)
    l1 = lambda n, j: 4.0 * n * n * np.sin(j * np.pi / (2 * n)) ** 2
    temp = sorted((-(l1(10, a) + l1(8, b) + l1(6, c)) / PR for a in range(1, 4) for b in range(4) for c in range(4)),
                  reverse=True)
    # the leading values at Gr = 0 are the temperature block's (the Stokes block lies further left here)
    assert np.allclose(lam[:4].real, temp[:4], rtol=1e-11, atol=0)
    assert np.all(np.abs(lam[:4].imag) <= 1e-9 * np.abs(lam[:4].real))


def test_symmetrise_projects_onto_the_symmetric_states():
    """oracle.sparse.symmetrise: its result has all three symmetry measures (Eqs. 7-9) at round-off and the
    velocity maps of Section 2 leave it unchanged; a symmetric steady state is a fixed point."""
    g = D.Grid(8, 7, 6, stretch=1.5, Pr=PR)
    q = _random_state(g, 9)
    qs = S.symmetrise(q)
    assert max(DG.symmetry_measures(g, qs[3])) <= 1e-14
    for img in (DG.sym_ref(qs), DG.sym_2d(qs), DG.sym_3d(qs)):
        for c in range(4):
            assert np.max(np.abs(img[c] - qs[c])) <= 1e-14
    qn, _ = S.newton_direct(g, 1.2e4, D.conduction_state(g), tol=1e-12)
    qq = S.symmetrise(qn)
    scale = max(float(np.max(np.abs(a))) for a in qn)
    assert max(float(np.max(np.abs(qq[c] - qn[c]))) for c in range(4)) <= 1e-10 * scale   # Section 2: ~1e-9
