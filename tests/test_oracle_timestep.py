"""Pins of the oracle's semi-implicit time step (oracle/timestep.py).

* Conduction at Gr = 0 is a fixed point (F = 0 exactly).
* At Gr = 0 about conduction a temperature eigenmode of the discrete Laplacian (uniform grid: Dirichlet
  sin(k pi (i + 1/2) / n) in x, Neumann cos(l pi (j + 1/2) / n) in y) decays by exactly 1 / (1 - dt mu) per
  step, mu = -(4 n_x^2 sin^2(k pi / 2 n_x) + 4 n_y^2 sin^2(l pi / 2 n_y)) / Pr, the backward-Euler factor of
  the closed-form eigenvalue, and no velocity appears (u = 0 removes convection; Gr = 0 buoyancy).
* One step agrees with the explicit step dt P F(q) up to O(dt^2): the difference shrinks fourfold when dt
  halves (the linearly implicit diffusion is a first-order perturbation of it).
* The velocity stays divergence free.
"""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle import timestep as TS
from oracle.projection import Projector
from paper_2210_08816_gb300 import seeded

PR = 0.71


def test_conduction_is_a_fixed_point():
    g = D.Grid(7, 6, 5, stretch=1.5, Pr=PR)
    q0 = D.conduction_state(g)
    q1 = TS.SemiImplicit(g, 0.0, 1e-2).step(q0)
    for c in range(4):
        assert np.max(np.abs(q1[c] - q0[c])) <= 1e-15


@pytest.mark.parametrize("kx,ly", [(1, 0), (2, 1), (3, 2)])
def test_temperature_eigenmode_decays_by_the_backward_euler_factor(kx, ly):
    nx, ny, nz, dt, eps = 10, 8, 6, 3e-3, 1e-2
    g = D.Grid(nx, ny, nz, stretch=0.0, Pr=PR)
    i, j = np.arange(nx) + 0.5, np.arange(ny) + 0.5
    mode = np.sin(kx * np.pi * i / nx)[None, None, :] * np.cos(ly * np.pi * j / ny)[None, :, None] * np.ones((nz, 1, 1))
    mu = -(4 * nx ** 2 * np.sin(kx * np.pi / (2 * nx)) ** 2 + 4 * ny ** 2 * np.sin(ly * np.pi / (2 * ny)) ** 2) / PR
    q = D.conduction_state(g)
    q[3] = q[3] + eps * mode
    ts = TS.SemiImplicit(g, 0.0, dt)
    for _ in range(3):
        q = ts.step(q)
    amp = eps / (1.0 - dt * mu) ** 3
    assert np.max(np.abs(q[3] - (1.0 - g.axes[0].xc)[None, None, :] - amp * mode)) <= 1e-13
    for c in range(3):
        assert np.max(np.abs(q[c])) <= 1e-14


def _state(g):
    q = D.from_api(g, seeded.normal_fields(61, g.shape, 2.0))
    q = Projector(g).full(q)
    q[3] = q[3] + (1.0 - g.axes[0].xc)[None, None, :]
    return q


def test_first_order_consistency_with_the_explicit_step():
    g = D.Grid(8, 7, 6, stretch=1.5, Pr=PR)
    Gr = 2e4
    q = _state(g)
    PF = Projector(g).full(D.residual_full(g, Gr, q))
    diffs = []
    for dt in (2e-5, 1e-5):
        q1 = TS.SemiImplicit(g, Gr, dt).step(q)
        diffs.append(max(float(np.max(np.abs(q1[c] - q[c] - dt * PF[c]))) for c in range(4)))
    assert 3.6 < diffs[0] / diffs[1] < 4.4, diffs


def test_velocity_stays_divergence_free():
    g = D.Grid(8, 7, 6, stretch=1.5, Pr=PR)
    q, ek, nu = TS.SemiImplicit(g, 5e4, 1e-4).run(_state(g), 4)
    scale = max(float(np.max(np.abs(q[c]))) for c in range(3))
    assert np.max(np.abs(D.divergence_full(g, q[:3]))) <= 1e-11 * scale / min(float(np.min(a.dx)) for a in g.axes)
    assert len(ek) == 5 and len(nu) == 5 and np.all(np.isfinite(ek)) and np.all(np.isfinite(nu))
