"""Host operands of the tensor-core pressure-solve passes (paper_2210_08816_gb300/csrc/host_tc.cpp) on the CPU.

The passes are the fast-diagonalisation solve of the SIMPLE-like projection (Section 1 methods paragraph,
Section 3) written for a mirror-symmetric grid: per axis a forward (cells -> modes) and a backward
(modes -> cells) transform, each two half-size matrices for the symmetric and antisymmetric modes, stored
as TF32 hi + FP32 lo.  Pins, from the definitions:
* every hi is a TF32 number (its 13 low mantissa bits are zero) and hi + lo restores the matrix to far
  below FP32 round-off;
* assembled to full size, the backward transform inverts the forward one, and diagonalises the 1D
  Neumann operator of the axis with the stored eigenvalues (the operator assembled from the library's own
  metric arrays, and the same eigenvalues as the library's full-size decomposition);
* the symmetric modes are even and the antisymmetric modes odd about the midplane;
* the per-step B blocks of the persistent pass hold exactly the hi / lo slabs of every K step, each row's
  16-byte chunks in the order the kernels' converters and MMAs read a 64-byte swizzled row (chunk c of row
  r at position c ^ ((r >> 1) & 3)), 256-byte aligned, tiling their region of the buffer without gaps.
"""
import ctypes as C

import numpy as np
import pytest

DP = C.POINTER(C.c_double)
LLP = C.POINTER(C.c_longlong)
FP = C.POINTER(C.c_float)


@pytest.fixture(scope="module")
def L(host_shim):
    f = host_shim.shim_tc_operands
    f.restype = C.c_longlong
    f.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, FP, C.c_longlong, LLP, LLP, LLP]
    host_shim.shim_tanh_faces.restype = None
    host_shim.shim_tanh_faces.argtypes = [C.c_int, C.c_double, DP]
    host_shim.shim_build_axis.restype = C.c_int
    host_shim.shim_build_axis.argtypes = [C.c_int, DP] + [DP] * 13
    return host_shim


def _operands(L, nx, ny, nz, s):
    n = L.shim_tc_operands(nx, ny, nz, s, None, 0, None, None, None)
    assert n > 0
    buf = np.zeros(n, dtype=np.float32)
    moff, loff, soff = (np.zeros(k, dtype=np.int64) for k in (24, 3, 6))
    got = L.shim_tc_operands(nx, ny, nz, s, buf.ctypes.data_as(FP), n, moff.ctypes.data_as(LLP),
                             loff.ctypes.data_as(LLP), soff.ctypes.data_as(LLP))
    assert got == n
    return buf, moff.reshape(3, 8), loff, soff.reshape(3, 2)


def _axis(L, n, s):
    f = np.zeros(n + 1)
    L.shim_tanh_faces(n, s, f.ctypes.data_as(DP))
    out = {k: np.zeros(n + 1) for k in ("idx", "idc", "wl", "wr")}
    out.update({k: np.zeros(n) for k in ("lam", "cd_lam", "fd_lam")})
    out.update({k: np.zeros((n, n)) for k in ("Einv", "E", "cd_Einv", "cd_E", "fd_Einv", "fd_E")})
    order = ["idx", "idc", "wl", "wr", "lam", "Einv", "E", "cd_lam", "cd_Einv", "cd_E", "fd_lam", "fd_Einv", "fd_E"]
    assert L.shim_build_axis(n, f.ctypes.data_as(DP), *[out[k].ctypes.data_as(DP) for k in order]) == 0
    return out


def _mat(buf, off, h):
    return buf[off:off + h * h].reshape(h, h)


def _full(buf, moff, d, n):
    """Full-size forward F (modes x cells) and backward E (cells x modes), modes [symmetric | antisymmetric],
    from hi + lo in FP64."""
    h = n // 2
    M = [_mat(buf, moff[d][k], h).astype(np.float64) for k in range(8)]
    Fs, Fa, Es, Ea = M[0] + M[1], M[2] + M[3], M[4] + M[5], M[6] + M[7]
    F, E = np.zeros((n, n)), np.zeros((n, n))
    k = np.arange(h)
    F[:h, k], F[:h, n - 1 - k] = Fs, Fs
    F[h:, k], F[h:, n - 1 - k] = Fa, -Fa
    E[k, :h], E[n - 1 - k, :h] = Es, Es
    E[k, h:], E[n - 1 - k, h:] = Ea, -Ea
    return F, E


def _neumann(a, n):
    Lm = np.zeros((n, n))
    for i in range(n):
        if i + 1 < n:
            Lm[i, i + 1] += a["idc"][i + 1] * a["idx"][i]
            Lm[i, i] -= a["idc"][i + 1] * a["idx"][i]
        if i >= 1:
            Lm[i, i - 1] += a["idc"][i] * a["idx"][i]
            Lm[i, i] -= a["idc"][i] * a["idx"][i]
    return Lm


GRIDS = [(32, 64, 96, 1.5), (128, 32, 32, 1.5), (64, 64, 64, 0.0), (256, 32, 224, 1.5)]


@pytest.mark.parametrize("nx,ny,nz,s", GRIDS)
def test_tf32_split(L, nx, ny, nz, s):
    buf, moff, _, _ = _operands(L, nx, ny, nz, s)
    for d, n in enumerate((nx, ny, nz)):
        h = n // 2
        for j in range(0, 8, 2):
            hi, lo = _mat(buf, moff[d][j], h), _mat(buf, moff[d][j + 1], h)
            assert np.all(hi.view(np.uint32) & np.uint32(0x1FFF) == 0)
            assert np.max(np.abs(lo)) <= 2.0 ** -11 * np.max(np.abs(hi))


@pytest.mark.parametrize("nx,ny,nz,s", GRIDS)
def test_transforms_invert_each_other_and_diagonalise_the_axis_operator(L, nx, ny, nz, s):
    buf, moff, loff, _ = _operands(L, nx, ny, nz, s)
    for d, n in enumerate((nx, ny, nz)):
        F, E = _full(buf, moff, d, n)
        lam = buf[loff[d]:loff[d] + n].astype(np.float64)
        assert np.max(np.abs(E @ F - np.eye(n))) <= 1e-9
        a = _axis(L, n, s)
        Lm = _neumann(a, n)
        scale = np.max(np.abs(Lm))
        assert np.max(np.abs(Lm @ E - E * lam)) <= 1e-6 * scale * np.max(np.abs(E))
        assert lam[0] == 0.0
        assert np.allclose(np.sort(lam), np.sort(a["lam"]), rtol=1e-6, atol=1e-6 * scale)
        h = n // 2
        assert np.all(np.diff(lam[:h]) <= 0) and np.all(np.diff(lam[h:]) <= 0)
        k = np.arange(h)
        assert np.array_equal(E[k, :h], E[n - 1 - k, :h]) and np.array_equal(E[k, h:], -E[n - 1 - k, h:])


@pytest.mark.parametrize("nx,ny,nz,s", GRIDS)
def test_persistent_pass_blocks_hold_the_swizzled_slabs(L, nx, ny, nz, s):
    buf, moff, loff, soff = _operands(L, nx, ny, nz, s)
    starts, ends = [], []
    for d, n in enumerate((nx, ny, nz)):
        h = n // 2
        nst = h // 16
        r = np.arange(h)[:, None]
        for direction in range(2):
            base = int(soff[d][direction])
            assert base % 64 == 0
            blk = buf[base:base + nst * 4 * h * 16].reshape(nst, 4, h, 4, 4)  # step, slab, row, chunk, float
            for m in range(4):
                M = _mat(buf, moff[d][4 * direction + m], h)
                for j in range(nst):
                    want = M[:, 16 * j:16 * j + 16].reshape(h, 4, 4)  # row, logical chunk, float
                    got = blk[j, m][np.arange(h)[:, None], np.arange(4)[None, :] ^ ((r >> 1) & 3)]
                    assert np.array_equal(got, want), (d, direction, m, j)
            starts.append(base)
            ends.append(base + nst * 4 * h * 16)
    order = np.argsort(starts)
    starts, ends = np.array(starts)[order], np.array(ends)[order]
    assert np.array_equal(starts[1:], ends[:-1])  # contiguous, no overlap
    assert ends[-1] == len(buf)
    ns = (nx, ny, nz)
    first = max(max(int(loff[d]) + ns[d], int(moff[d][7]) + (ns[d] // 2) ** 2) for d in range(3))
    assert starts[0] >= first  # after every matrix and eigenvalue array
