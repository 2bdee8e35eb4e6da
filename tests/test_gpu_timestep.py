"""The time-dependent path (Section 4.2.3) through the C-ABI against the oracle.

* fv_diagnostics: E_kin (Eq. 12) and Nu (Eq. 13) of a seeded state against oracle.diagnostics, 1e-12.
* fv_time_step: five semi-implicit steps (FP64) against oracle.timestep on the same seeded state, every field
  at 1e-10 of its size, and the E_kin / Nu histories at 1e-10 (the step inverts I - dt L once per field and
  projects once: a few FP64 transforms of rounding per step, compounded over five steps).
"""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle import diagnostics as DG
from oracle import timestep as TS
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


def _state(og, seed=71, sigma=3.0):
    q = D.from_api(og, seeded.normal_fields(seed, og.shape, sigma))
    q = Projector(og).full(q)
    q[3] = q[3] + (1.0 - og.axes[0].xc)[None, None, :]
    return q


def _dev(og, q):
    return torch.tensor(np.stack(D.to_api(og, q)), dtype=torch.float64, device="cuda").contiguous().view(-1)


@pytest.mark.parametrize("shape,stretch", [((12, 10, 8), 1.5), ((16, 16, 16), 0.0)])
def test_diagnostics_match_oracle(fv, shape, stretch):
    og = D.Grid(*shape, stretch=stretch, Pr=PR)
    g = fv.Grid(*shape, stretch=stretch, Pr=PR)
    q = _state(og)
    ek, nu = fv.fv_diagnostics(g, _dev(og, q))
    assert ek == pytest.approx(DG.kinetic_energy(og, q), rel=1e-12)
    assert nu == pytest.approx(DG.nusselt_hot(og, q[3]), rel=1e-12)
    g.close()


@pytest.mark.parametrize("shape,stretch,Gr,dt", [((12, 10, 8), 1.5, 5e4, 1e-4), ((20, 16, 12), 0.0, 2e5, 5e-5)])
def test_time_steps_match_oracle(fv, shape, stretch, Gr, dt):
    og = D.Grid(*shape, stretch=stretch, Pr=PR)
    g = fv.Grid(*shape, stretch=stretch, Pr=PR)
    q0 = _state(og)
    qd = _dev(og, q0)
    ek, nu = fv.fv_time_step(g, Gr, dt, 5, qd)
    torch.cuda.synchronize()
    q_ref, ek_ref, nu_ref = TS.SemiImplicit(og, Gr, dt).run(q0, 5)
    got = qd.view(4, *og.shape).cpu().numpy()
    ref = D.to_api(og, q_ref)
    for c in range(4):
        assert np.max(np.abs(got[c] - ref[c])) <= 1e-10 * max(1.0, float(np.max(np.abs(ref[c])))), c
    assert np.allclose(ek, ek_ref, rtol=1e-10, atol=0)
    assert np.allclose(nu, nu_ref, rtol=1e-10, atol=0)
    assert ek[-1] != ek[0]   # the state moved
    g.close()
