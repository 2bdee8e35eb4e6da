"""The library's host construction of a grid axis (paper_2210_08816_gb300/csrc/host_grid.cpp) on the CPU.

* Faces: the tanh-stretched mirrored grid equals the oracle's faces (the same reading of Section 4.1's
  "stretched near the borders"), is mirror-symmetric exactly, runs from 0 to 1 and is uniform at s = 0.
* Metrics: widths, centre spacings and interpolation weights equal the oracle's Axis.
* The 1D decompositions of the pressure solve and of the Newton preconditioner reproduce their operators
  (L E = E diag(lam), Einv E = I), and on a uniform grid take the textbook eigenvalues: Neumann
  -(2/h)^2 sin^2(k pi / 2n), k = 0 .. n-1 (the constant vector first, with lam exactly 0), face-centred
  Dirichlet the same expression for k = 1 .. n-1.
"""
import ctypes as C

import numpy as np
import pytest

import oracle.discretisation as D

DP = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def L(host_shim):
    host_shim.shim_tanh_faces.restype = None
    host_shim.shim_tanh_faces.argtypes = [C.c_int, C.c_double, DP]
    host_shim.shim_build_axis.restype = C.c_int
    host_shim.shim_build_axis.argtypes = [C.c_int, DP] + [DP] * 13
    return host_shim


def _faces(L, n, s):
    f = np.zeros(n + 1)
    L.shim_tanh_faces(n, s, f.ctypes.data_as(DP))
    return f


def _axis(L, xf):
    n = len(xf) - 1
    out = {k: np.zeros(n + 1) for k in ("idx", "idc", "wl", "wr")}
    out.update({k: np.zeros(n) for k in ("lam", "cd_lam", "fd_lam")})
    out.update({k: np.zeros((n, n)) for k in ("Einv", "E", "cd_Einv", "cd_E", "fd_Einv", "fd_E")})
    order = ["idx", "idc", "wl", "wr", "lam", "Einv", "E", "cd_lam", "cd_Einv", "cd_E", "fd_lam", "fd_Einv", "fd_E"]
    x = np.ascontiguousarray(xf, dtype=np.float64)
    st = L.shim_build_axis(n, x.ctypes.data_as(DP), *[out[k].ctypes.data_as(DP) for k in order])
    return st, out


@pytest.mark.parametrize("n,s", [(8, 0.0), (12, 1.5), (33, 1.5), (100, 1.5), (256, 1.5), (17, 2.5)])
def test_faces_match_the_oracle_and_are_mirror_symmetric(L, n, s):
    f = _faces(L, n, s)
    assert np.max(np.abs(f - D.faces(n, s))) <= 1e-15
    assert f[0] == 0.0 and f[-1] == 1.0
    assert np.all(np.diff(f) > 0.0)
    k = np.arange(n // 2 + 1)
    assert np.array_equal(f[n - k], 1.0 - f[k])  # the upper half is the mirrored lower half, bit for bit
    if s == 0.0:
        assert np.max(np.abs(f - np.arange(n + 1) / n)) <= 1e-16


@pytest.mark.parametrize("n,s", [(7, 1.5), (32, 1.5), (100, 1.5)])
def test_metrics_match_the_oracle_axis(L, n, s):
    ax = D.Axis(n, s)
    st, a = _axis(L, ax.xf)
    assert st == 0
    assert np.allclose(a["idx"][:n], 1.0 / ax.dx, rtol=1e-14, atol=0)
    assert np.allclose(a["idc"][1:n], 1.0 / ax.dc, rtol=1e-13, atol=0)
    assert a["idc"][0] == pytest.approx(2.0 / ax.dx[0], rel=1e-15)
    assert a["idc"][n] == pytest.approx(2.0 / ax.dx[-1], rel=1e-15)
    assert np.allclose(a["wl"][1:n], ax.wl, rtol=1e-14, atol=0)
    assert np.allclose(a["wr"][1:n], ax.wr, rtol=1e-14, atol=0)


def _neumann(a, n):
    """(L u)_i = [(u_{i+1} - u_i) idc[i+1] - (u_i - u_{i-1}) idc[i]] idx[i] with zero flux through the walls."""
    Lm = np.zeros((n, n))
    for i in range(n):
        if i + 1 < n:
            Lm[i, i + 1] += a["idc"][i + 1] * a["idx"][i]
            Lm[i, i] -= a["idc"][i + 1] * a["idx"][i]
        if i >= 1:
            Lm[i, i - 1] += a["idc"][i] * a["idx"][i]
            Lm[i, i] -= a["idc"][i] * a["idx"][i]
    return Lm


def _dirichlet_cells(a, n):
    """As the Neumann operator, with Dirichlet walls half a cell away (idc[0], idc[n] reach the wall)."""
    Lm = _neumann(a, n)
    Lm[0, 0] -= a["idc"][0] * a["idx"][0]
    Lm[n - 1, n - 1] -= a["idc"][n] * a["idx"][n - 1]
    return Lm


def _dirichlet_faces(a, n):
    """Faces p = 1 .. n-1: (L u)_p = [(u_{p+1} - u_p) idx[p] - (u_p - u_{p-1}) idx[p-1]] idc[p], u_0 = u_n = 0;
    slot 0 (the wall) is the identity's dummy mode."""
    Lm = np.zeros((n, n))
    Lm[0, 0] = -1.0
    for p in range(1, n):
        Lm[p, p] = -(a["idx"][p] + a["idx"][p - 1]) * a["idc"][p]
        if p + 1 < n:
            Lm[p, p + 1] = a["idx"][p] * a["idc"][p]
        if p - 1 >= 1:
            Lm[p, p - 1] = a["idx"][p - 1] * a["idc"][p]
    return Lm


@pytest.mark.parametrize("n,s", [(6, 0.0), (24, 1.5), (64, 1.5)])
def test_decompositions_reproduce_their_operators(L, n, s):
    st, a = _axis(L, D.faces(n, s))
    assert st == 0
    for lam, E, Einv, op in [(a["lam"], a["E"], a["Einv"], _neumann(a, n)),
                             (a["cd_lam"], a["cd_E"], a["cd_Einv"], _dirichlet_cells(a, n)),
                             (a["fd_lam"], a["fd_E"], a["fd_Einv"], _dirichlet_faces(a, n))]:
        scale = np.max(np.abs(op))
        assert np.max(np.abs(Einv @ E - np.eye(n))) <= 1e-12 * n
        assert np.max(np.abs(op @ E - E * lam)) <= 1e-11 * scale * np.max(np.abs(E))
    assert a["lam"][0] == 0.0 and np.all(np.diff(a["lam"]) <= 0.0) and np.all(a["lam"][1:] < 0.0)


@pytest.mark.parametrize("n", [5, 16, 40])
def test_uniform_grid_takes_the_textbook_eigenvalues(L, n):
    st, a = _axis(L, np.arange(n + 1) / n)
    assert st == 0
    k = np.arange(n)
    closed = -(2.0 * n * np.sin(k * np.pi / (2 * n))) ** 2
    assert np.max(np.abs(np.sort(a["lam"]) - np.sort(closed))) <= 1e-11 * (2.0 * n) ** 2
    fd = np.sort(a["fd_lam"][1:])
    assert np.max(np.abs(fd - np.sort(closed[1:]))) <= 1e-11 * (2.0 * n) ** 2


def test_non_increasing_faces_are_refused(L):
    st, _ = _axis(L, np.array([0.0, 0.5, 0.5, 1.0]))
    assert st != 0


def test_only_mirror_symmetric_axes_take_the_tensor_core_passes(L):
    # the tensor-core passes split every 1D eigenproblem into symmetric and antisymmetric halves: an axis
    # qualifies only if its faces are their own mirror image about 1/2
    f = L.shim_mirror_symmetric
    f.restype, f.argtypes = C.c_int, [C.c_int, DP]

    def sym(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return f(len(x) - 1, x.ctypes.data_as(DP)) == 1

    for n, s in [(32, 0.0), (64, 1.5), (256, 1.5), (33, 2.0)]:
        assert sym(_faces(L, n, s))
    one_sided = (np.exp(2.0 * np.arange(65) / 64) - 1.0) / (np.exp(2.0) - 1.0)  # clustered at x = 0 only
    assert not sym(one_sided)
    x = _faces(L, 64, 1.5)
    x[10] += 1e-9
    assert not sym(x)
    x = _faces(L, 64, 1.5)
    x[10] = np.nextafter(x[10], 1.0)  # one unit of round-off stays within the tolerance
    assert sym(x)
