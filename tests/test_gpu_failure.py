"""Failure detection on the GPU without a fault: the give-up path of the bounded device-side waits.

Every mbarrier wait in the library's kernels (the TMA plane ring of the J.v stencils, the pipeline of the
tcgen05 pressure-solve passes) polls a bounded number of times.  fv_set_wait_limit(g, 0) makes each such
wait give up at its first poll: the kernel records a code in the handle's error word, stops issuing work,
lets the bulk copies and tensor-core operations it has started complete, frees its tensor memory and
returns.  The call then reports FV_ETIMEOUT (fv_sync, or any call that reads a scalar back), and the next
call with the default limit on the same handle computes the oracle's result again.  Nothing here faults,
traps or hangs: every copy the kernels wait for is a legitimate one that completes.
"""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle.projection import Projector
from paper_2210_08816_gb300 import seeded

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
PR = 0.71


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_08816_gb300 import build
    build.build()
    from paper_2210_08816_gb300 import fv as _fv
    _fv.lib()
    return _fv


def _inputs(og, prec):
    q = D.from_api(og, seeded.normal_fields(81, og.shape, 0.5))
    q = Projector(og).full(q)
    q[3] = q[3] + (1.0 - og.axes[0].xc)[None, None, :]
    qa = D.to_api(og, q)
    va = D.to_api(og, D.from_api(og, seeded.normal_fields(82, og.shape)))
    if prec == "fp32":
        qa = [a.astype(np.float32).astype(np.float64) for a in qa]
        va = [a.astype(np.float32).astype(np.float64) for a in va]
    return qa, va


def _oracle(og, Gr, sigma, qa, va):
    qf, vf = D.from_api(og, qa), D.from_api(og, va)
    J = D.jvp_full(og, Gr, qf, vf)
    r = Projector(og).full([J[c] - sigma * vf[c] for c in range(4)])
    return D.to_api(og, [r[c] + sigma * vf[c] for c in range(4)])


def _rel(got, ref):
    return max(float(np.max(np.abs(got[c] - ref[c]))) / max(float(np.max(np.abs(ref[c]))), 1e-300)
               for c in range(4))


# (shape, precision): two-cell TMA stencil + tcgen05 passes; one-cell TMA stencil (nx % 64 != 0) + SIMT
# passes; FP64 one-cell TMA stencil
CASES = [((64, 64, 64), "fp32"), ((96, 48, 40), "fp32"), ((64, 32, 24), "fp64")]


@pytest.mark.parametrize("shape,prec", CASES)
def test_give_up_reports_timeout_and_the_handle_recovers(fv, shape, prec):
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    p = fv.FV_FP32 if prec == "fp32" else fv.FV_FP64
    dt = torch.float32 if prec == "fp32" else torch.float64
    Gr, sigma = 2.0e6, -500.0
    qa, va = _inputs(og, prec)
    q = torch.tensor(np.stack(qa), dtype=dt, device="cuda").contiguous().view(-1)
    v = torch.tensor(np.stack(va), dtype=dt, device="cuda").contiguous().view(-1)
    out = torch.empty_like(v)
    assert fv.fv_sync(g) == fv.FV_OK
    fv.fv_set_wait_limit(g, 0)
    fv.fv_jvp_project(g, p, Gr, sigma, q, v, out)
    assert fv.fv_sync(g) == fv.FV_ETIMEOUT
    assert fv.fv_sync(g) == fv.FV_OK          # the report clears the error word
    # a call that reads a scalar back reports the same
    with pytest.raises(fv.FvError) as e:
        fv.fv_jvp_project_lincomb(g, p, Gr, sigma, q, v, None, 1.0, 0.0, 0.0, out, want_norm=True)
    assert e.value.status == fv.FV_ETIMEOUT
    # default limit: the same handle computes the oracle's result
    fv.fv_set_wait_limit(g, -1)
    out.zero_()
    fv.fv_jvp_project(g, p, Gr, sigma, q, v, out)
    assert fv.fv_sync(g) == fv.FV_OK
    got = out.view(4, *og.shape).double().cpu().numpy()
    tol = 5e-5 if prec == "fp32" else 1e-12
    assert _rel([got[c] for c in range(4)], _oracle(og, Gr, sigma, qa, va)) <= tol
    g.close()
