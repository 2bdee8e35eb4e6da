"""Pins of the oracle's F and J.v against things other than themselves.

* Gr = 0 conduction (T = 1 - x, u = 0) is an exact steady state on any grid
  (Section 2, Eqs. 4-6); at Gr > 0 the only non-zero residual is the buoyancy
  Gr (1 - x) e_z.
* Manufactured smooth fields: interior truncation error of every term of
  Eqs. 1-2 (convection, diffusion, buoyancy, thermal diffusion 1/Pr) decays as
  h^2 against the analytic PDE operator (sympy).
* Closed-form eigenvectors of the diffusion part with the wall closures of
  Section 2 (no-slip; Eq. 4 Dirichlet; Eqs. 5-6 Neumann).
* F is quadratic, so central differences of F reproduce J.v exactly.
* The three symmetries of Section 2 commute with P F and with J; on a grid without mirror symmetry the
  reflection y -> 1 - y maps F and J.v on the grid to F and J.v on the reflected grid.
"""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle import diagnostics as S
from oracle.projection import Projector
from paper_2210_08816_gb300 import seeded

PR = 0.71


def _rand_full(g, seed, sigma=1.0):
    return D.from_api(g, seeded.normal_fields(seed, g.shape, sigma))


def _scale(g):
    h = min(float(a.dx.min()) for a in g.axes)
    return 1.0 / (h * h)


def test_grid_faces_mirrored_and_stretched():
    for n in (7, 12, 100, 256):
        for s in (0.0, 1.5):
            xf = D.faces(n, s)
            assert xf[0] == 0.0 and xf[-1] == 1.0
            assert np.all(np.diff(xf) > 0)
            lo = np.arange(n // 2 + 1)
            assert np.array_equal(xf[n - lo], 1.0 - xf[lo])     # upper half is the mirrored lower half
            dx = np.diff(xf)
            assert np.allclose(dx[::-1], dx, rtol=1e-13, atol=0)
    dx = np.diff(D.faces(256, 1.5))
    # tanh law with s = 1.5: cells shrink toward the walls
    assert dx[0] < dx[128] and dx.max() / dx.min() == pytest.approx(
        np.cosh(1.5) ** 2, rel=2e-2)   # sech^2 slope ratio of the tanh law


@pytest.mark.parametrize("shape,stretch", [((12, 10, 8), 0.0), ((7, 5, 3), 1.5), ((16, 16, 16), 1.5)])
def test_conduction_is_exact_steady_state_at_Gr0(shape, stretch):
    g = D.Grid(*shape, stretch=stretch, Pr=PR)
    F = D.residual_full(g, 0.0, D.conduction_state(g))
    tol = 1e-13 * _scale(g)
    for c in range(4):
        assert np.max(np.abs(F[c])) <= tol


def test_conduction_buoyancy_only_at_positive_Gr():
    g = D.Grid(9, 6, 7, stretch=1.5, Pr=PR)
    Gr = 2.5e5
    F = D.residual_full(g, Gr, D.conduction_state(g))
    xc = g.axes[0].xc
    expect = np.broadcast_to(Gr * (1.0 - xc)[None, None, :], (g.nz - 1, g.ny, g.nx))
    assert np.allclose(F[2][1:-1], expect, rtol=1e-13, atol=0)
    for c in (0, 1):
        assert np.max(np.abs(F[c])) == 0.0
    assert np.max(np.abs(F[3])) <= 1e-13 * _scale(g)


# --------------------------------------------------------------------------- manufactured solution
def _mms_functions(Gr):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    pi = sp.pi
    A = 5
    u = A * sp.sin(pi * x) * sp.sin(pi * y) * sp.sin(pi * z) * (1 + x + y / 2)
    v = A * sp.sin(2 * pi * x) * sp.sin(pi * y) * sp.sin(pi * z) * (1 + z)
    w = A * sp.sin(pi * x) * sp.sin(pi * y) * sp.sin(2 * pi * z) * (sp.Rational(1, 2) + y)
    T = 1 - x + sp.Rational(1, 5) * sp.sin(pi * x) * sp.cos(pi * y) * sp.cos(2 * pi * z) \
        + sp.Rational(1, 10) * x * (1 - x) * sp.cos(pi * y)
    vel = (u, v, w)
    X = (x, y, z)
    lap = lambda f: sum(sp.diff(f, s, 2) for s in X)
    conv = lambda f: sum(sp.diff(vel[d] * f, X[d]) for d in range(3))
    Fu = -conv(u) + lap(u)
    Fv = -conv(v) + lap(v)
    Fw = -conv(w) + lap(w) + Gr * T
    FT = -conv(T) + lap(T) / sp.Float(PR)
    lam = lambda f: sp.lambdify((x, y, z), f, "numpy")
    return [lam(f) for f in (u, v, w, T)], [lam(f) for f in (Fu, Fv, Fw, FT)]


def _sample(g, fns):
    gx, gy, gz = g.axes
    pts = [(gx.xf, gy.xc, gz.xc), (gx.xc, gy.xf, gz.xc), (gx.xc, gy.xc, gz.xf), (gx.xc, gy.xc, gz.xc)]
    out = []
    for f, (px, py, pz) in zip(fns, pts):
        Z, Y, X = np.meshgrid(pz, py, px, indexing="ij")
        out.append(np.broadcast_to(f(X, Y, Z), Z.shape).astype(np.float64).copy())
    return out


def _one_sided(n, a):
    """Faces clustered towards x = 0 only (no mirror symmetry): x_f = (e^(a i/n) - 1) / (e^a - 1)."""
    xf = np.expm1(a * np.arange(n + 1) / n) / np.expm1(a)
    xf[0], xf[-1] = 0.0, 1.0
    return xf


@pytest.mark.parametrize("stretch", [0.0, 1.5, "one-sided"])
def test_residual_second_order_against_pde(stretch):
    # the one-sided grid has no mirror symmetry, so a metric index taken from the wrong end of an axis
    # (which a mirror-symmetric grid cannot show) breaks the convergence
    Gr = 40.0
    fields, exact = _mms_functions(Gr)
    errs = []
    for n in (16, 32, 64):
        if stretch == "one-sided":
            g = D.Grid(n, n, n, Pr=PR, xyz_faces=(_one_sided(n, 1.2), _one_sided(n, -0.8), _one_sided(n, 0.6)))
        else:
            g = D.Grid(n, n, n, stretch=stretch, Pr=PR)
        q = _sample(g, fields)
        for c in range(3):                       # no-slip: the sampled walls are ~1e-16; make them exact
            ax = 2 - c
            sl = [slice(None)] * 3
            sl[ax] = 0
            q[c][tuple(sl)] = 0.0
            sl[ax] = -1
            q[c][tuple(sl)] = 0.0
        F = D.residual_full(g, Gr, q)
        ref = _sample(g, exact)
        e = []
        for c in range(4):
            core = (slice(2, -2),) * 3           # away from the walls (one-sided closures)
            e.append(np.max(np.abs(F[c][core] - ref[c][core])) / np.max(np.abs(ref[c][core])))
        errs.append(e)
    errs = np.array(errs)
    assert np.all(errs[-1] < 5e-3)
    ratios = errs[:-1] / errs[1:]
    if stretch == "one-sided":   # the place of the largest error moves between levels: judge two halvings
        assert np.all(ratios > 2.5) and np.all(errs[0] / errs[-1] > 10.0), (errs, ratios)
    else:
        assert np.all(ratios > 3.0), (errs, ratios)


# --------------------------------------------------------------------------- diffusion closed forms
def _lam1(n, k):
    return 4.0 * n * n * np.sin(k * np.pi / (2 * n)) ** 2


def test_velocity_diffusion_closed_form_eigenvectors():
    nx, ny, nz = 10, 8, 6
    g = D.Grid(nx, ny, nz, stretch=0.0, Pr=PR)
    zero = [np.zeros(g.full_shape(c)) for c in range(3)] + [np.zeros(g.shape)]
    gx, gy, gz = g.axes
    for (a, b, c) in [(1, 1, 1), (3, 2, 5), (9, 8, 1)]:
        # u on x-faces (vertex-type Dirichlet in x), cell-type Dirichlet in y and z
        Z, Y, X = np.meshgrid(gz.xc, gy.xc, gx.xf, indexing="ij")
        u = np.sin(a * np.pi * X) * np.sin(b * np.pi * Y) * np.sin(c * np.pi * Z)
        u[:, :, 0] = u[:, :, -1] = 0.0
        v = [u, np.zeros(g.full_shape(1)), np.zeros(g.full_shape(2)), np.zeros(g.shape)]
        J = D.jvp_full(g, 0.0, zero, v)
        lam = -(_lam1(nx, a) + _lam1(ny, b) + _lam1(nz, c))
        assert np.max(np.abs(J[0] - lam * u)) <= 1e-12 * abs(lam)
        assert max(np.max(np.abs(J[k])) for k in (1, 2, 3)) == 0.0


def test_temperature_diffusion_closed_form_eigenvectors():
    nx, ny, nz = 10, 8, 6
    g = D.Grid(nx, ny, nz, stretch=0.0, Pr=PR)
    zero = [np.zeros(g.full_shape(c)) for c in range(3)] + [np.zeros(g.shape)]
    gx, gy, gz = g.axes
    Z, Y, X = np.meshgrid(gz.xc, gy.xc, gx.xc, indexing="ij")
    for (a, b, c) in [(1, 0, 0), (2, 1, 3), (10, 7, 5)]:
        T = np.sin(a * np.pi * X) * np.cos(b * np.pi * Y) * np.cos(c * np.pi * Z)   # Eq. 4 Dirichlet, Eqs. 5-6 Neumann
        v = [np.zeros(g.full_shape(k)) for k in range(3)] + [T]
        J = D.jvp_full(g, 0.0, zero, v)
        lam = -(_lam1(nx, a) + _lam1(ny, b) + _lam1(nz, c)) / PR
        assert np.max(np.abs(J[3] - lam * T)) <= 1e-12 * abs(lam)


# --------------------------------------------------------------------------- J.v
@pytest.mark.parametrize("shape,stretch", [((12, 10, 8), 1.5), ((7, 5, 3), 0.0)])
def test_jvp_equals_central_difference_of_quadratic_F(shape, stretch):
    g = D.Grid(*shape, stretch=stretch, Pr=PR)
    q = _rand_full(g, 11)
    q[3] = q[3] + (1.0 - g.axes[0].xc)[None, None, :]
    v = _rand_full(g, 12)
    Gr = 3.0e4
    J = D.jvp_full(g, Gr, q, v)
    for eps in (1e-3, 0.37):
        Fp = D.residual_full(g, Gr, [q[c] + eps * v[c] for c in range(4)])
        Fm = D.residual_full(g, Gr, [q[c] - eps * v[c] for c in range(4)])
        for c in range(4):
            fd = (Fp[c] - Fm[c]) / (2 * eps)
            assert np.max(np.abs(fd - J[c])) <= 1e-10 * np.max(np.abs(J[c]))


def test_convective_heat_flux_is_conservative():
    g = D.Grid(9, 7, 5, stretch=1.5, Pr=PR)
    a = _rand_full(g, 21)
    b = _rand_full(g, 22)
    C = D.convection(g, a, b)
    gx, gy, gz = g.axes
    V = gz.dx[:, None, None] * gy.dx[None, :, None] * gx.dx[None, None, :]
    assert abs(np.sum(V * C[3])) <= 1e-13 * np.sum(V * np.abs(C[3]))


# --------------------------------------------------------------------------- symmetries
@pytest.mark.parametrize("sym", [S.sym_ref, S.sym_2d, S.sym_3d])
def test_symmetries_commute_with_PF_and_J(sym):
    g = D.Grid(10, 8, 6, stretch=1.5, Pr=PR)
    P = Projector(g)
    q = P.full(_rand_full(g, 31))
    q[3] = q[3] + (1.0 - g.axes[0].xc)[None, None, :]
    v = P.full(_rand_full(g, 32))
    Gr = 5.0e4
    a = P.full(D.residual_full(g, Gr, sym(q)))
    b = sym(P.full(D.residual_full(g, Gr, q)), affine=False)
    for c in range(4):
        assert np.max(np.abs(a[c] - b[c])) <= 1e-12 * np.max(np.abs(b[c]))
    a = D.jvp_full(g, Gr, sym(q), sym(v, affine=False))
    b = sym(D.jvp_full(g, Gr, q, v), affine=False)
    for c in range(4):
        assert np.max(np.abs(a[c] - b[c])) <= 1e-12 * np.max(np.abs(b[c]))


def _reflect_y(q):
    """The mirror image y -> 1 - y of full arrays: every field reversed along y (numpy axis 1), v negated."""
    out = [np.flip(a, axis=1).copy() for a in q]
    out[1] = -out[1]
    return out


def test_reflection_of_an_asymmetric_grid_reflects_F_and_J():
    # y -> 1 - y maps the problem onto itself (Section 2: adiabatic y walls, buoyancy along z).  On a grid
    # whose y faces are not symmetric the reflected field lives on the reflected grid, and F and J.v there
    # must be the reflections of F and J.v here: every wall closure and interpolation weight of the y
    # direction enters at both ends, so one taken from the wrong end of the axis breaks the relation
    n = (9, 8, 7)
    xf, yf, zf = _one_sided(n[0], 0.9), _one_sided(n[1], 1.3), _one_sided(n[2], -0.7)
    g = D.Grid(*n, Pr=PR, xyz_faces=(xf, yf, zf))
    gr = D.Grid(*n, Pr=PR, xyz_faces=(xf, 1.0 - yf[::-1], zf))
    q = _rand_full(g, 41)
    q[3] = q[3] + (1.0 - g.axes[0].xc)[None, None, :]
    v = _rand_full(g, 42)
    Gr = 3.0e4
    pairs = [(D.residual_full(gr, Gr, _reflect_y(q)), _reflect_y(D.residual_full(g, Gr, q))),
             (D.jvp_full(gr, Gr, _reflect_y(q), _reflect_y(v)), _reflect_y(D.jvp_full(g, Gr, q, v)))]
    for a, b in pairs:
        for c in range(4):
            assert np.max(np.abs(a[c] - b[c])) <= 1e-12 * np.max(np.abs(b[c])), c


def test_layout_round_trip():
    g = D.Grid(5, 4, 3)
    api = seeded.normal_fields(5, g.shape)
    full = D.from_api(g, api)
    back = D.to_api(g, full)
    for c in range(3):
        ax = 2 - c
        sl = [slice(None)] * 3
        sl[ax] = slice(1, None)
        assert np.array_equal(back[c][tuple(sl)], api[c][tuple(sl)])
        sl[ax] = 0
        assert np.all(back[c][tuple(sl)] == 0.0)
    assert np.array_equal(D.unpack(g, D.pack(full))[3], full[3])
    assert D.pack(full).size == D.n_unknowns(g)
