"""The Chebyshev filter's confocal ellipses (paper_2210_08816_gb300/csrc/host_cheb.cpp) on the CPU.

The Chebyshev-preconditioned Arnoldi iteration (Section 1 methods paragraph and its ref. 21) damps the
unwanted part of the spectrum with T_deg((z - d)/c), whose modulus grows like level(z)^deg, level(z) = |w|
for z - d = c (w + 1/w) / 2: the level sets are the ellipses with foci d +- c.  Pins, all from that
definition: the level is (a + b)/|c| on the ellipse of semi-axes a, b (real foci for a > b, imaginary for
b > a), xi + sqrt(xi^2 - 1) on the real axis, 1 on the focal segment, the radius for circles; the right end
of an ellipse is d + a; for unwanted values filling a real interval and a wanted value to its right the
best ellipse is the interval itself (Chebyshev's optimality on an interval), with the closed-form rate;
and on random Ritz sets the selection follows its stated rule over its candidate grid.
"""
import ctypes as C
import math

import numpy as np
import pytest

D = C.c_double
DP = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def L(host_shim):
    host_shim.shim_ellipse_level.restype = D
    host_shim.shim_ellipse_level.argtypes = [D, D, D, D]
    host_shim.shim_ellipse_right_end.restype = D
    host_shim.shim_ellipse_right_end.argtypes = [D, D, D]
    host_shim.shim_best_ellipse.restype = None
    host_shim.shim_best_ellipse.argtypes = [C.c_int, DP, DP, C.c_int, DP, DP, DP, DP, DP]
    return host_shim


def _best(L, wanted, unwanted):
    w = np.array(wanted, dtype=complex)
    u = np.array(unwanted, dtype=complex)
    wr, wi = np.ascontiguousarray(w.real), np.ascontiguousarray(w.imag)
    ur, ui = np.ascontiguousarray(u.real), np.ascontiguousarray(u.imag)
    d, c2, rate = D(), D(), D()
    L.shim_best_ellipse(len(w), wr.ctypes.data_as(DP), wi.ctypes.data_as(DP), len(u), ur.ctypes.data_as(DP),
                        ui.ctypes.data_as(DP), C.byref(d), C.byref(c2), C.byref(rate))
    return d.value, c2.value, rate.value


@pytest.mark.parametrize("a,b", [(5.0, 3.0), (40.0, 1.0), (3.0, 5.0), (1.0, 90.0)])
def test_level_is_constant_on_an_ellipse(L, a, b):
    d = -7.0
    c2 = a * a - b * b  # real foci for a > b, imaginary for b > a
    expect = (a + b) / math.sqrt(abs(c2))
    for th in np.linspace(0.0, 2.0 * math.pi, 13):
        z = complex(d + a * math.cos(th), b * math.sin(th))
        assert L.shim_ellipse_level(z.real, z.imag, d, c2) == pytest.approx(expect, rel=1e-12)
    assert L.shim_ellipse_right_end(d, c2, expect) == pytest.approx(d + a, rel=1e-12, abs=1e-12)


def test_level_on_the_real_axis_and_the_focal_segment(L):
    d, c = 3.0, 2.0
    for x in (5.5, 9.0, 100.0):
        xi = (x - d) / c
        assert L.shim_ellipse_level(x, 0.0, d, c * c) == pytest.approx(xi + math.sqrt(xi * xi - 1), rel=1e-13)
        assert L.shim_ellipse_level(2 * d - x, 0.0, d, c * c) == pytest.approx(xi + math.sqrt(xi * xi - 1), rel=1e-13)
    for x in np.linspace(d - c, d + c, 9):
        assert L.shim_ellipse_level(x, 0.0, d, c * c) == pytest.approx(1.0, abs=1e-7)


def test_circles(L):
    assert L.shim_ellipse_level(3.0, 4.0, 0.0, 0.0) == pytest.approx(5.0, rel=1e-15)
    assert L.shim_ellipse_right_end(-2.0, 0.0, 5.0) == pytest.approx(3.0, rel=1e-15)


def test_interval_of_unwanted_values_gives_the_interval_itself(L):
    unwanted = list(np.linspace(-100.0, -10.0, 19))
    d, c2, rate = _best(L, [-1.0], unwanted)
    assert d == pytest.approx(-55.0, abs=1e-12)
    assert c2 == pytest.approx(45.0 ** 2, rel=1e-12)
    xi = 54.0 / 45.0
    assert rate == pytest.approx(xi + math.sqrt(xi * xi - 1.0), rel=1e-6)


def _scan(L, wanted, unwanted):
    """The selection rule written out over the same candidate grid: centres at 0.2 .. 0.8 of the unwanted
    real span (13), c^2 from -1 to 1 times max(half-extent^2, max |Im|^2) (41); the best ratio among
    candidates whose right end stays left of every wanted real part, else the best of all."""
    ure = [z.real for z in unwanted]
    amin, amax = min(ure), max(ure)
    bmax = max(abs(z.imag) for z in unwanted)
    wleft = min(z.real for z in wanted)
    span = max(amax - amin, 1e-12 * max(1.0, abs(amax)))
    best_ok, best_any = -1.0, -1.0
    for a in range(13):
        d = amin + (0.2 + 0.05 * a) * span
        a0 = max(amax - d, d - amin)
        for t in range(41):
            c2 = (-1.0 + 0.05 * t) * max(a0 * a0, bmax * bmax)
            lu = max(L.shim_ellipse_level(z.real, z.imag, d, c2) for z in unwanted)
            lw = min(L.shim_ellipse_level(z.real, z.imag, d, c2) for z in wanted)
            rate = lw / lu if lu > 0 else 1e300
            best_any = max(best_any, rate)
            if L.shim_ellipse_right_end(d, c2, lu) <= wleft:
                best_ok = max(best_ok, rate)
    return (best_ok, True) if best_ok >= 0.0 else (best_any, False)


@pytest.mark.parametrize("seed", range(6))
def test_selection_follows_its_rule_on_random_ritz_sets(L, seed):
    rng = np.random.default_rng(seed)
    nu = 12
    unwanted = list(rng.uniform(-3000, -50, nu) + 1j * rng.uniform(-800, 800, nu))
    wanted = list(rng.uniform(-40, 5, 3) + 1j * rng.uniform(-300, 300, 3))
    d, c2, rate = _best(L, wanted, unwanted)
    lu = max(L.shim_ellipse_level(z.real, z.imag, d, c2) for z in unwanted)
    lw = min(L.shim_ellipse_level(z.real, z.imag, d, c2) for z in wanted)
    expect, qualified = _scan(L, wanted, unwanted)
    assert rate == pytest.approx(lw / lu, rel=1e-12)
    assert rate == pytest.approx(expect, rel=1e-12)
    if qualified:  # then the chosen ellipse keeps every wanted value to its right
        assert L.shim_ellipse_right_end(d, c2, lu) <= min(z.real for z in wanted)
