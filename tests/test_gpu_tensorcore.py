"""Tensor-core (tcgen05, 3 x TF32) pressure-solve passes: FP32 projection and fused J.v + projection
against the FP64 oracle on grids whose every dimension is a multiple of 32 in [32, 256] (the sizes that
take the tensor-core path): cubic, non-cubic, and 64 x 96 x 224 whose x pass has P = 224 * 96 = 21504
rows = 168 tiles of 128 while its z pass has P = 96 * 64 = 6144; other grids use the SIMT passes."""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle.projection import Projector
from paper_2210_08816_gb300 import seeded

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
PR = 0.71
TOL32 = 5e-5   # same bound as the SIMT FP32 path: six transforms of ~sqrt(n) u each


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_08816_gb300 import build
    build.build()
    from paper_2210_08816_gb300 import fv as _fv
    _fv.lib()
    return _fv


def dev(api):
    return torch.tensor(np.stack(api), dtype=torch.float32, device="cuda").contiguous().view(-1)


def host(t, shape):
    a = t.view(4, *shape).double().cpu().numpy()
    return [a[c] for c in range(4)]


def rel(a, b):
    return max(float(np.max(np.abs(a[c] - b[c]))) / max(float(np.max(np.abs(b[c]))), 1e-300) for c in range(4))


def r32(api):
    return [a.astype(np.float32).astype(np.float64) for a in api]


@pytest.mark.parametrize("shape,stretch", [((64, 64, 64), 1.5), ((96, 160, 32), 1.5), ((32, 32, 96), 0.0),
                                           ((64, 96, 224), 1.5), ((128, 128, 128), 1.5)])
def test_tensorcore_projection_fp32(fv, shape, stretch):
    og = D.Grid(*shape, stretch=stretch, Pr=PR)
    g = fv.Grid(*shape, stretch=stretch, Pr=PR)
    v = r32(D.to_api(og, D.from_api(og, seeded.normal_fields(61, og.shape))))
    ref = Projector(og).api(v)
    t = dev(v)
    it, div = fv.fv_project(g, fv.FV_FP32, t, max_it=1, want_div=True)
    assert div <= 1e-4
    assert rel(host(t, og.shape), ref) <= TOL32


@pytest.mark.parametrize("shape", [(64, 64, 64), (96, 160, 32)])
def test_tensorcore_fused_fp32(fv, shape):
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q = D.from_api(og, seeded.normal_fields(62, og.shape, 0.5))
    q[3] = q[3] + (1.0 - og.axes[0].xc)[None, None, :]
    q = r32(D.to_api(og, q))
    v = r32(D.to_api(og, D.from_api(og, seeded.normal_fields(63, og.shape))))
    Gr, sigma = 3.0e6, -400.0
    P = Projector(og)
    qf, vf = D.from_api(og, q), D.from_api(og, v)
    J = D.jvp_full(og, Gr, qf, vf)
    A = P.full([J[c] - sigma * vf[c] for c in range(4)])
    ref = D.to_api(og, [A[c] + sigma * vf[c] for c in range(4)])
    out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    fv.fv_jvp_project(g, fv.FV_FP32, Gr, sigma, dev(q), dev(v), out)
    assert rel(host(out, og.shape), ref) <= TOL32
