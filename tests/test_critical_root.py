"""The root iteration behind fv_critical_gr (Section 4.1: the critical Gr is where the real part of the
tracked eigenvalue crosses zero), run on host functions through fv_critical_root; no GPU.

Pins: a linear function is solved by one secant step; a bracketed smooth crossing converges to the
requested tolerance; before a bracket every secant step is at most twice the previous spacing; the
Illinois halving makes a strongly convex crossing converge where plain false position stalls (plain false
position is written out below and shown not to converge in the same number of steps); a failing or
non-finite evaluation ends the iteration with its status; bad options are refused.
"""
import ctypes as C
import math

import pytest

pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fv():
    from paper_2210_08816_gb300 import build
    build.build()
    from paper_2210_08816_gb300 import fv as _fv
    _fv.lib()
    return _fv


def _opts(fv, a, b, tol=1e-7, max_iter=16):
    c = fv.fv_critical_default_opts()
    c.gr_a, c.gr_b, c.tol, c.max_iter = a, b, tol, max_iter
    return c


def _history(rep):
    return [rep.gr[i] for i in range(rep.evaluations)], [rep.re[i] for i in range(rep.evaluations)]


def test_linear_function_is_solved_by_one_secant_step(fv):
    st, rep = fv.fv_critical_root(_opts(fv, 2.0e5, 2.5e5), lambda g: (g - 3.0e5) / 1.0e5)
    assert st == fv.FV_OK
    assert rep.evaluations == 3
    assert rep.gr_cr == pytest.approx(3.0e5, rel=1e-12)
    assert abs(rep.lam_re) <= 1e-12


def test_bracketed_crossing_converges_to_the_tolerance(fv):
    x0, w, im = 4.2e5, 3.0e4, 481.0
    st, rep = fv.fv_critical_root(_opts(fv, 3.9e5, 4.4e5), lambda g: complex(math.tanh((g - x0) / w), im))
    assert st == fv.FV_OK
    assert rep.gr_cr == pytest.approx(x0, rel=1e-7)
    assert rep.lam_im == im
    assert rep.omega_scaled == pytest.approx(im / math.sqrt(rep.gr_cr), rel=1e-15)
    grs, res = _history(rep)
    assert grs[:2] == [3.9e5, 4.4e5] and grs[-1] == rep.gr_cr and res[-1] == rep.lam_re


def test_secant_steps_are_limited_until_a_sign_change(fv):
    x0 = 6.0e5
    f = lambda g: math.tanh((g - x0) / 1.0e5)  # noqa: E731
    st, rep = fv.fv_critical_root(_opts(fv, 1.0e5, 1.2e5, max_iter=30), f)
    assert st == fv.FV_OK
    assert rep.gr_cr == pytest.approx(x0, rel=1e-7)
    grs, res = _history(rep)
    for i in range(2, len(grs)):
        if any(r > 0.0 for r in res[:i]):
            break  # bracketed from here on
        assert abs(grs[i] - grs[i - 1]) <= 2.0 * abs(grs[i - 1] - grs[i - 2]) * (1 + 1e-12), (i, grs)
    assert max(grs) < 1.0e6  # no runaway step from the nearly flat start


def _plain_false_position(f, a, b, steps):
    fa, fb = f(a), f(b)
    for _ in range(steps):
        x = b - fb * (b - a) / (fb - fa)
        fx = f(x)
        if fx * fb < 0.0:
            a, fa = b, fb
        b, fb = x, fx
    return b


def test_illinois_halving_converges_where_false_position_stalls(fv):
    f = lambda g: (g / 1.0e5) ** 8 - 1.0  # noqa: E731  (root 1e5, strongly convex on the bracket)
    st, rep = fv.fv_critical_root(_opts(fv, 0.5e5, 2.0e5, max_iter=16), f)
    assert st == fv.FV_OK
    assert rep.gr_cr == pytest.approx(1.0e5, rel=1e-7)
    assert rep.evaluations <= 18
    assert abs(_plain_false_position(f, 0.5e5, 2.0e5, 16) - 1.0e5) > 1e3


def test_no_crossing_ends_at_the_cap(fv):
    st, rep = fv.fv_critical_root(_opts(fv, 1.0e5, 2.0e5, max_iter=6), lambda g: 1.0 + (g / 1.0e6) ** 2)
    assert st == fv.FV_ENOCONV
    assert 2 <= rep.evaluations <= 8
    assert all(r > 0.0 for r in _history(rep)[1])


def test_a_failing_evaluation_ends_the_iteration_with_its_status(fv):
    calls = []

    def raw(gr, ctx, re, im):
        calls.append(gr)
        if len(calls) == 3:
            return fv.FV_ENOCONV
        re[0], im[0] = (gr - 3.0e5) ** 2 / 1e10 - 1.0, 0.0
        return fv.FV_OK

    cb = fv.TRACKED_FN(raw)
    rep = fv.fv_critical_report()
    st = fv.lib().fv_critical_root(C.byref(_opts(fv, 1.0e5, 1.5e5)), cb, None, C.byref(rep))
    assert st == fv.FV_ENOCONV and rep.status == fv.FV_ENOCONV
    assert rep.evaluations == 2 and rep.gr_cr == 1.5e5 and len(calls) == 3

    def boom(g):
        if g > 2.0e5:
            raise ValueError("evaluation failed")
        return (g - 3.0e5) / 1.0e5

    with pytest.raises(ValueError):
        fv.fv_critical_root(_opts(fv, 1.0e5, 1.5e5), boom)

    with pytest.raises(fv.FvError) as e:
        fv.fv_critical_root(_opts(fv, 1.0e5, 1.5e5), lambda g: float("nan") if g > 1.6e5 else g - 3e5)
    assert e.value.status == fv.FV_ENAN


@pytest.mark.parametrize("a,b,tol,max_iter", [(1e5, 1e5, 1e-7, 16), (0.0, 1e5, 1e-7, 16), (1e5, 2e5, 0.0, 16),
                                              (1e5, 2e5, 1e-7, 39), (1e5, 2e5, 1e-7, -1)])
def test_bad_options_are_refused(fv, a, b, tol, max_iter):
    with pytest.raises(fv.FvError) as e:
        fv.fv_critical_root(_opts(fv, a, b, tol, max_iter), lambda g: g - 1.5e5)
    assert e.value.status == fv.FV_EINVAL
