"""fv_dot_noalloc: the inner product for callers that cannot allocate device memory.

Such callers (allocation-free real-time loops, fixed memory budgets, memory owned by another pool)
cannot create an fv_grid handle, whose construction allocates workspace.  The no-allocation entry
point keeps its partial sums in a static device array instead.  Checked through the C-ABI against
the existing handle-based fv_dot on the same vectors, twice in a row (the shared scratch keeps the
previous call's contents), within the inner-product tolerance the other tests use.  This file is
collected last so that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2210_08816_gb300 import seeded

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_08816_gb300 import build
    build.build()
    from paper_2210_08816_gb300 import fv as _fv
    _fv.lib()
    return _fv


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_noalloc_dot_matches_handle_dot_twice(fv, prec_name):
    nx, ny, nz = 96, 80, 72          # 4*N = 2.2M elements: 9 blocks of the static scratch, ragged tail
    g = fv.Grid(nx, ny, nz)
    prec = fv.FV_FP64 if prec_name == "fp64" else fv.FV_FP32
    dt = torch.float64 if prec_name == "fp64" else torch.float32
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call, (sa, sb) in enumerate([(21, 22), (23, 24)]):
        a = torch.tensor(np.stack(seeded.normal_fields(sa, (nz, ny, nx))), dtype=dt, device="cuda").view(-1)
        b = torch.tensor(np.stack(seeded.normal_fields(sb, (nz, ny, nx))), dtype=dt, device="cuda").view(-1)
        ref = fv.fv_dot(g, prec, a, b)
        fv.fv_dot_noalloc(prec, a, b, res)
        torch.cuda.synchronize()
        got = float(res.item())
        scale = float(torch.sum(torch.abs(a.double() * b.double())).item())
        assert abs(got - ref) <= 1e-12 * scale, (call, got, ref)


def test_noalloc_dot_rejects_bad_sizes(fv):
    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = fv.lib()
    import ctypes as C
    st = L.fv_dot_noalloc(0, 4096 * (1 << 18) + 1, C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()),
                          C.c_void_p(res.data_ptr()), None)
    assert st == fv.FV_EINVAL
    assert L.fv_dot_noalloc(0, 0, C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()), C.c_void_p(res.data_ptr()),
                            None) == fv.FV_EINVAL
    assert L.fv_dot_noalloc(5, 8, C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()), C.c_void_p(res.data_ptr()),
                            None) == fv.FV_EINVAL


def test_noalloc_dot_more_blocks_than_the_finishing_threads(fv):
    """FP32 vectors of 1100 * 2^18 elements (1.15 GB each): 1100 partial sums, more than the finishing
    kernel's 1024 threads, so its strided loop runs; every slot is reduced (checked against a float64 sum
    of the same products), on two calls in a row."""
    n = 1100 * (1 << 18)
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    gen = torch.Generator(device="cuda")
    for call, seed in enumerate((5, 6)):
        gen.manual_seed(seed)
        a = torch.randn(n, dtype=torch.float32, device="cuda", generator=gen)
        b = torch.randn(n, dtype=torch.float32, device="cuda", generator=gen)
        ref = sum(float(torch.dot(a[i:i + (1 << 26)].double(), b[i:i + (1 << 26)].double()).item())
                  for i in range(0, n, 1 << 26))
        scale = sum(float(torch.sum(torch.abs(a[i:i + (1 << 26)].double() * b[i:i + (1 << 26)].double())).item())
                    for i in range(0, n, 1 << 26))
        fv.fv_dot_noalloc(fv.FV_FP32, a, b, res)
        torch.cuda.synchronize()
        got = float(res.item())
        assert abs(got - ref) <= 1e-12 * scale, (call, got, ref)
        del a, b
    torch.cuda.empty_cache()


def test_noalloc_dot_rejects_host_memory(fv):
    """A host pointer (or one the current device cannot dereference) is refused before any launch."""
    import ctypes as C
    h = np.zeros(8)
    dres = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = fv.lib()
    hp = C.c_void_p(h.ctypes.data)
    assert L.fv_dot_noalloc(0, 8, hp, hp, C.c_void_p(dres.data_ptr()), None) == fv.FV_EINVAL
    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert L.fv_dot_noalloc(0, 8, C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()), hp, None) == fv.FV_EINVAL
