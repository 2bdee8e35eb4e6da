"""Pins of the oracle's D, G and projection P (Section 3: divergence-free Krylov vectors).

* D reproduces the analytic divergence of fields that are quadratic along
  their own axis (exact midpoint rule); G is exact on linear potentials
  (stretched grid) and quadratic ones (uniform grid).
* DG on a uniform grid has the closed-form Neumann spectrum
  -(4/h^2) sin^2(k pi / 2n) with cosine eigenvectors.
* P is the projector onto null(D) along range(G): D P v = 0, P^2 = P,
  P G phi = 0, P v = v for divergence-free v, and P is self-adjoint in the
  face-volume inner product; the FDM and CG solves agree.
"""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle.projection import Projector, cg_solve, FDM, laplacian, neumann_matrix
from paper_2210_08816_gb300 import seeded


def _rand_full(g, seed):
    return D.from_api(g, seeded.normal_fields(seed, g.shape))


def _mesh(g, which):
    gx, gy, gz = g.axes
    pts = {"u": (gx.xf, gy.xc, gz.xc), "v": (gx.xc, gy.xf, gz.xc), "w": (gx.xc, gy.xc, gz.xf),
           "c": (gx.xc, gy.xc, gz.xc)}[which]
    Z, Y, X = np.meshgrid(pts[2], pts[1], pts[0], indexing="ij")
    return X, Y, Z


def _one_sided(n, a):
    """Faces clustered towards one wall only (no mirror symmetry): x_f = (e^(a i/n) - 1) / (e^a - 1)."""
    xf = np.expm1(a * np.arange(n + 1) / n) / np.expm1(a)
    xf[0], xf[-1] = 0.0, 1.0
    return xf


def _grid(shape, stretch):
    if stretch == "one-sided":
        return D.Grid(*shape, xyz_faces=(_one_sided(shape[0], 1.5), _one_sided(shape[1], -1.0),
                                         _one_sided(shape[2], 0.7)))
    return D.Grid(*shape, stretch=stretch)


@pytest.mark.parametrize("stretch", [0.0, 1.5, "one-sided"])
def test_divergence_exact_on_own_axis_quadratics(stretch):
    g = _grid((9, 7, 6), stretch)
    X, Y, Z = _mesh(g, "u")
    u = X * (1 - X) * (1 + Y * Y + Z)           # zero on the x-walls, quadratic in x
    X, Y, Z = _mesh(g, "v")
    v = Y * (1 - Y) * np.cos(X + 2 * Z)
    X, Y, Z = _mesh(g, "w")
    w = Z * (1 - Z) * (X - Y) ** 3
    u[:, :, [0, -1]] = 0.0
    v[:, [0, -1], :] = 0.0
    w[[0, -1], :, :] = 0.0
    X, Y, Z = _mesh(g, "c")
    exact = (1 - 2 * X) * (1 + Y * Y + Z) + (1 - 2 * Y) * np.cos(X + 2 * Z) + (1 - 2 * Z) * (X - Y) ** 3
    assert np.max(np.abs(D.divergence_full(g, [u, v, w]) - exact)) <= 1e-12


@pytest.mark.parametrize("stretch", [1.5, "one-sided"])
def test_gradient_exact_on_linear_and_uniform_quadratic(stretch):
    g = _grid((8, 6, 5), stretch)
    X, Y, Z = _mesh(g, "c")
    G = D.gradient_full(g, 2.0 * X - 3.0 * Y + 0.5 * Z)
    assert np.allclose(G[0][:, :, 1:-1], 2.0, rtol=1e-12)
    assert np.allclose(G[1][:, 1:-1, :], -3.0, rtol=1e-12)
    assert np.allclose(G[2][1:-1], 0.5, rtol=1e-12)
    gu = D.Grid(8, 6, 5, stretch=0.0)
    X, Y, Z = _mesh(gu, "c")
    G = D.gradient_full(gu, X * X + Y * Z)
    Xu, Yu, Zu = _mesh(gu, "u")
    assert np.allclose(G[0][:, :, 1:-1], (2 * Xu)[:, :, 1:-1], rtol=0, atol=1e-12)
    for c, ax in ((0, 2), (1, 1), (2, 0)):     # walls carry no gradient
        sl = [slice(None)] * 3
        sl[ax] = 0
        assert np.all(G[c][tuple(sl)] == 0.0)


def test_neumann_laplacian_closed_form():
    n = 11
    g = D.Grid(n, n, n).axes[0]
    A = neumann_matrix(g)
    lam = np.sort(np.linalg.eigvals(A).real)[::-1]
    expect = np.sort(-4.0 * n * n * np.sin(np.arange(n) * np.pi / (2 * n)) ** 2)[::-1]
    assert np.allclose(lam, expect, rtol=1e-12, atol=1e-9)
    for k in (0, 3, 10):
        e = np.cos(k * np.pi * g.xc)
        assert np.allclose(A @ e, -4.0 * n * n * np.sin(k * np.pi / (2 * n)) ** 2 * e, atol=1e-9)


@pytest.mark.parametrize("shape,stretch", [((10, 8, 6), 1.5), ((7, 5, 3), 0.0), ((12, 12, 12), 1.5)])
def test_projection_invariants(shape, stretch):
    g = D.Grid(*shape, stretch=stretch)
    P = Projector(g)
    v = _rand_full(g, 41)
    pv = P.full(v)
    vnorm = max(np.max(np.abs(v[c])) for c in range(3))
    scale = vnorm / min(float(a.dx.min()) for a in g.axes)
    assert np.max(np.abs(D.divergence_full(g, pv[:3]))) <= 1e-12 * scale     # D P v = 0
    ppv = P.full(pv)
    for c in range(3):
        assert np.max(np.abs(ppv[c] - pv[c])) <= 1e-13 * vnorm                # P^2 = P
    assert np.array_equal(pv[3], v[3])                                        # T untouched
    phi = seeded.normal(42, 0, int(np.prod(g.shape))).reshape(g.shape)
    Gphi = D.gradient_full(g, phi)
    pg = P.full(Gphi + [np.zeros(g.shape)])
    gn = max(np.max(np.abs(Gphi[c])) for c in range(3))
    for c in range(3):
        assert np.max(np.abs(pg[c])) <= 1e-12 * gn                            # P G phi = 0
    # self-adjoint in the face-volume inner product <a,b>_W = sum_f vol_f a_f b_f
    gx, gy, gz = g.axes
    W = [gz.dx[:, None, None] * gy.dx[None, :, None] * gx.dc[None, None, :],
         gz.dx[:, None, None] * gy.dc[None, :, None] * gx.dx[None, None, :],
         gz.dc[:, None, None] * gy.dx[None, :, None] * gx.dx[None, None, :]]
    a, b = _rand_full(g, 43), _rand_full(g, 44)
    pa, pb = P.full(a), P.full(b)
    ip = lambda x, y: sum(float(np.sum(W[c] * D.interior_velocity(x, c) * D.interior_velocity(y, c)))
                          for c in range(3))
    assert abs(ip(pa, b) - ip(a, pb)) <= 1e-12 * abs(ip(pa, pb))


def test_fdm_agrees_with_cg():
    g = D.Grid(9, 7, 6, stretch=1.5)
    v = _rand_full(g, 51)
    rhs = D.divergence_full(g, v[:3])
    phi_f = FDM(g).solve(rhs)
    phi_c = cg_solve(g, rhs, tol=1e-15)
    assert np.max(np.abs(laplacian(g, phi_f) - rhs)) <= 1e-11 * np.max(np.abs(rhs))
    Gf, Gc = D.gradient_full(g, phi_f), D.gradient_full(g, phi_c)
    for c in range(3):
        assert np.max(np.abs(Gf[c] - Gc[c])) <= 1e-11 * np.max(np.abs(Gf[c]))
