"""The library's host linear algebra (paper_2210_08816_gb300/csrc/host_linalg.cpp) on the CPU.

These routines carry the pressure solve's 1D eigen-decompositions (symmetric tridiagonal QR), the Arnoldi
iteration's Hessenberg eigenproblem and Ritz vectors (Section 1 methods paragraph, Section 3), the Rayleigh-
Ritz reduction, BiCGstab(2)'s small systems and GMRES's least-squares problem.  They are compiled here with
a test-only C wrapper (tests/host_shim.cpp) and checked against what fixes them independently:
matrices built with a known spectrum (orthogonal similarity of a block-diagonal matrix), the defining
identities (T Q = Q Lambda, Q^T Q = I, A = Q H Q^T, H y = lambda y), and SciPy / NumPy's LAPACK routines.
"""
import ctypes as C

import numpy as np
import pytest

sl = pytest.importorskip("scipy.linalg")

DP = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def L(host_shim):
    lib = host_shim
    i = C.c_int
    for name, res, args in [("shim_tridiag_eig", i, [i, DP, DP, DP]),
                            ("shim_hessenberg_eigvals", i, [i, DP, DP, DP]),
                            ("shim_hessenberg_eigvec", i, [i, DP, C.c_double, C.c_double, DP]),
                            ("shim_hessenberg_reduce", None, [i, DP, DP]),
                            ("shim_hessenberg_lstsq", None, [i, DP, i, C.c_double, DP, DP]),
                            ("shim_dense_solve", i, [i, DP, DP])]:
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(DP)


def _tridiag(L, d, e):
    n = len(d)
    dd, ee, Q = d.copy(), (e.copy() if n > 1 else np.zeros(1)), np.zeros((n, n))
    assert L.shim_tridiag_eig(n, _p(dd), _p(ee), _p(Q)) == 1
    return dd, Q


def _known_spectrum(rng, pairs, reals):
    """A real matrix with eigenvalues a +- ib (pairs) and the reals, by a random orthogonal similarity of a
    block-diagonal matrix, then its Hessenberg form (SciPy); returns (H, exact eigenvalues)."""
    blocks = [np.array([[a, b], [-b, a]]) for a, b in pairs] + [np.array([[r]]) for r in reals]
    B = sl.block_diag(*blocks)
    m = B.shape[0]
    Qr, _ = np.linalg.qr(rng.standard_normal((m, m)))
    H = sl.hessenberg(Qr @ B @ Qr.T)
    H = np.ascontiguousarray(np.triu(H, -1))
    lam = [complex(a, b) for a, b in pairs] + [complex(a, -b) for a, b in pairs] + [complex(r) for r in reals]
    return H, np.array(lam)


def _match(computed, exact):
    """Largest distance from each exact eigenvalue to its partner, pairing greedily by distance."""
    left = list(computed)
    worst = 0.0
    for z in exact:
        k = int(np.argmin([abs(z - c) for c in left]))
        worst = max(worst, abs(z - left.pop(k)))
    return worst


@pytest.mark.parametrize("n", [1, 2, 3, 16, 128, 257])
def test_tridiagonal_eigendecomposition(L, n):
    rng = np.random.default_rng(100 + n)
    d, e = rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))
    lam, Q = _tridiag(L, d, e)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nrm = max(1.0, np.linalg.norm(T, 2))
    assert np.max(np.abs(np.sort(lam) - sl.eigh_tridiagonal(d, e, eigvals_only=True))) <= 1e-13 * nrm * n
    assert np.linalg.norm(T @ Q - Q * lam) <= 1e-13 * nrm * n
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * n


def test_tridiagonal_with_nearly_degenerate_pairs(L):
    # Wilkinson's W21+: eigenvalue pairs that agree to ~1e-14 relative, like the wall-localised pairs of a
    # stretched grid's 1D operator; the vectors must still come out orthonormal.
    d = np.abs(np.arange(21.0) - 10.0)
    e = np.ones(20)
    lam, Q = _tridiag(L, d, e)
    assert np.max(np.abs(np.sort(lam) - sl.eigh_tridiagonal(d, e, eigvals_only=True))) <= 1e-13 * 11
    assert np.linalg.norm(Q.T @ Q - np.eye(21)) <= 1e-12


@pytest.mark.parametrize("m", [1, 2, 9, 60, 200])
def test_hessenberg_eigenvalues_of_a_known_spectrum(L, m):
    rng = np.random.default_rng(m)
    npair = m // 3
    pairs = [(rng.uniform(-500, 10), rng.uniform(1, 900)) for _ in range(npair)]
    reals = list(rng.uniform(-3000, 5, m - 2 * npair))
    H, lam = _known_spectrum(rng, pairs, reals)
    re, im = np.zeros(m), np.zeros(m)
    assert L.shim_hessenberg_eigvals(m, _p(H), _p(re), _p(im)) == 1
    # a normal matrix: every eigenvalue is perfectly conditioned
    assert _match(re + 1j * im, lam) <= 1e-12 * np.linalg.norm(H, 2) * m
    # real input: the computed set is closed under conjugation
    assert _match(re - 1j * im, lam) <= 1e-12 * np.linalg.norm(H, 2) * m


def test_hessenberg_eigenvalues_of_a_nonnormal_matrix_match_lapack(L):
    rng = np.random.default_rng(7)
    m = 40
    H = np.ascontiguousarray(np.triu(rng.standard_normal((m, m)), -1))
    re, im = np.zeros(m), np.zeros(m)
    assert L.shim_hessenberg_eigvals(m, _p(H), _p(re), _p(im)) == 1
    assert _match(re + 1j * im, np.linalg.eigvals(H)) <= 1e-9 * np.linalg.norm(H, 2)
    assert abs(re.sum() - np.trace(H)) <= 1e-11 * np.linalg.norm(H, 2) * m


def test_hessenberg_eigenvectors_by_inverse_iteration(L):
    rng = np.random.default_rng(11)
    H, lam = _known_spectrum(rng, [(-5.0, 40.0), (-60.0, 3.0), (-1.0, 1e3)], [-2.0, -2.5, -700.0])
    m = H.shape[0]
    nrm = np.linalg.norm(H, 2)
    for z in lam:
        y = np.zeros(2 * m)
        assert L.shim_hessenberg_eigvec(m, _p(H), z.real, z.imag, _p(y)) == 1
        v = y[0::2] + 1j * y[1::2]
        assert np.linalg.norm(v) > 0.0
        assert np.linalg.norm(H @ v - z * v) <= 1e-12 * nrm * np.linalg.norm(v) * m


@pytest.mark.parametrize("m", [1, 2, 5, 60])
def test_householder_reduction_to_hessenberg(L, m):
    rng = np.random.default_rng(200 + m)
    A0 = rng.standard_normal((m, m))
    A, Q = A0.copy(), np.zeros((m, m))
    L.shim_hessenberg_reduce(m, _p(A), _p(Q))
    assert np.all(np.tril(A, -2) == 0.0)
    assert np.linalg.norm(Q @ A @ Q.T - A0) <= 1e-14 * np.linalg.norm(A0) * m
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 1e-14 * m


@pytest.mark.parametrize("j", [1, 3, 30])
def test_gmres_least_squares(L, j):
    rng = np.random.default_rng(300 + j)
    ld = j + 4  # a leading dimension wider than the matrix, as in the GMRES workspace
    Hfull = np.zeros((j + 1, ld))
    Hfull[:, :j] = np.triu(rng.standard_normal((j + 1, j)), -1)
    beta = 2.5
    y, resid = np.zeros(j), np.zeros(1)
    L.shim_hessenberg_lstsq(j, _p(Hfull), ld, beta, _p(y), _p(resid))
    H = Hfull[:, :j]
    rhs = np.zeros(j + 1)
    rhs[0] = beta
    yref = np.linalg.lstsq(H, rhs, rcond=None)[0]
    assert np.linalg.norm(y - yref) <= 1e-11 * max(1.0, np.linalg.norm(yref))
    assert resid[0] == pytest.approx(np.linalg.norm(H @ y - rhs), rel=1e-10, abs=1e-13)


def test_dense_solve_pivots_and_refuses_singular_systems(L):
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    x = np.array([1.0, -2.0, 0.5])
    b = A @ x
    assert L.shim_dense_solve(3, _p(A), _p(b)) == 1  # needs a row exchange at the first step
    assert np.max(np.abs(b - x)) <= 1e-15 * 8
    rng = np.random.default_rng(5)
    A = rng.standard_normal((10, 10)) + 10 * np.eye(10)
    x = rng.standard_normal(10)
    b = A @ x
    assert L.shim_dense_solve(10, _p(A), _p(b)) == 1
    assert np.max(np.abs(b - x)) <= 1e-13
    S = np.array([[1.0, 2.0], [2.0, 4.0]])  # rank 1: the second pivot is exactly 0 after elimination
    b = np.array([1.0, 1.0])
    assert L.shim_dense_solve(2, _p(S), _p(b)) == 0
